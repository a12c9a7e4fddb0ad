// C ABI of the capillary-bridge library: context life cycle, set-up, stepping under a captured
// CUDA graph, read-out. Declared in include/cbl.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cbl.h"
#include "cbl_dev.cuh"

using namespace cbl;

namespace cbl {
thread_local int g_launch_share = 1;
}

// sets the share of the GPU for the launches of this host thread while in scope
struct LaunchShare {
  int keep;
  explicit LaunchShare(int n) : keep(g_launch_share) { g_launch_share = n < 1 ? 1 : n; }
  ~LaunchShare() { g_launch_share = keep; }
};

struct cbl_ctx {
  cbl_params p;
  cbl_allocator alloc;
  bool user_alloc = false;
  cudaStream_t s = nullptr;
  bool own_stream = false;
  // side branch of the captured step (near-solid collision and repulsion run beside the bulk
  // collision): its stream and the fork / join events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int branches = 1;  // 0: the step graph is one chain
  Lat lat;
  int prec = 1;
  size_t elem = 4;
  PhysParams pp;
  LbmOps ops;  // launchers of the context's velocity set
  void *fa = nullptr, *fb = nullptr, *psi = nullptr;
  void* nbuf = nullptr;  // (rho, psi) of the fluid cells next to a solid, written by the collision
  uint16_t* flags = nullptr;
  double *diag_rho = nullptr, *diag_vel = nullptr, *dense = nullptr, *popbuf = nullptr;
  std::vector<BodyDev> hb;
  BodyDev* db = nullptr;
  double* arena = nullptr;
  long long arena_n = 0;
  int max_tile = 0;
  double *acc = nullptr, *last = nullptr, *volacc = nullptr, *scratch = nullptr;
  double* fsum = nullptr;      // per body: running sums of the total force and torque (6 doubles)
  long long fsum_steps = 0;    // steps summed into fsum since its last reset
  double* rtab = nullptr;  // per body and axis: minimum-image offsets of the tile coordinates
  int* mbox = nullptr;     // per body: member record (box lo[3], hi[3], largest squared distance; MBOX_N ints)
  int Lmax = 1;            // longest tile side
  double* mass_part = nullptr;
  unsigned n_mass_part = 0;
  int* blist = nullptr;  // fluid cells next to a solid (capacity: the sum of the tile sizes)
  // accumulating pass (lbm_variant 2): the bulk collision also sums the next step's density; psi
  // alternates between psi and psi2 with the parity, rhop holds the regions' edge partial sums
  int acc_pass = 0;
  int acc_ty = 8;          // y extent of its regions (8 or 16; x extent 32)
  int acc_sz_req = 0;      // requested z extent of a region (0 = derived)
  int acc_sz = 0;          // z extent in use
  int acc_attr_ty = 0;     // region depth whose kernel has its shared-memory limit set
  void *psi2 = nullptr, *rhop = nullptr;
  bool psi_valid = false;  // psi of the current step is in place (else a whole-lattice density pass first)
  int fused_tz = 0;      // > 0: the density and the bulk collision run as one fused pass (k_fused)
  int fused_tz_req = 0;  // requested z extent of a fused block (0 = derived)
  int fused_ty = 8;      // y extent of a fused block's consumer tile (4 or 8; x extent 32)
  int block_x = 32;      // x extent of the split kernels' 128-thread blocks
  double tile_tail = 2.5;  // cells of room for the advection tail in each body tile
  int node_priority = 1;   // 1: the step graph keeps the side stream's priority on its kernels
  StepState* st = nullptr;
  bool ready = false;
  long long t = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // live timing of the bulk collision inside the replayed step graph ("kernel_events" option): two
  // event-record nodes bracket its launch; before each replay they are pointed at the next pair of
  // a ring of events, so the pairs of the last steps can be read back after the replays
  int kev = 0;
  cudaEvent_t kev_cap[2] = {nullptr, nullptr};
  cudaGraphNode_t kev_node[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> kev_ring;  // 2 * KEV_RING events
  long long kev_steps = 0;            // replays recorded by the last cbl_step
  std::vector<void*> allocs;
  std::string err;
};

static thread_local std::string g_err;

static cbl_status fail(cbl_ctx* c, cbl_status s, const std::string& m) {
  if (c) c->err = m;
  else g_err = m;
  return s;
}

static cbl_status cuda_check(cbl_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CBL_OK;
  return fail(c, CBL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(call)                                            \
  do {                                                      \
    cbl_status _s = cuda_check(ctx, (call), #call);         \
    if (_s != CBL_OK) return _s;                            \
  } while (0)

static void* dalloc(cbl_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (c->user_alloc) {
    p = c->alloc.alloc(bytes, c->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) c->allocs.push_back(p);
  return p;
}

static void dfree_all(cbl_ctx* c) {
  for (void* p : c->allocs) {
    if (c->user_alloc) c->alloc.free(p, c->alloc.user);
    else cudaFree(p);
  }
  c->allocs.clear();
}

extern "C" {

const char* cbl_last_error(const cbl_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

cbl_status cbl_create(const cbl_params* params, const cbl_allocator* alloc, cbl_ctx** out) {
  if (!params || !out) return fail(nullptr, CBL_ERR_ARG, "params and out must not be NULL");
  const cbl_params& p = *params;
  if (p.nx < 4 || p.ny < 4 || p.nz < 4) return fail(nullptr, CBL_ERR_ARG, "lattice sides must be >= 4");
  if (p.q != 19 && p.q != 27) return fail(nullptr, CBL_ERR_UNSUPPORTED, "velocity sets: D3Q19 or D3Q27");
  {
    const double vals[] = {p.tau, p.G, p.rho0, p.ext_force[0], p.ext_force[1], p.ext_force[2], p.mobility, p.eta,
                           p.sigma_sf, p.sigma_ss, p.e0, p.rc, p.solid_threshold, p.member_threshold};
    for (double v : vals)
      if (!std::isfinite(v)) return fail(nullptr, CBL_ERR_ARG, "parameters must be finite");
  }
  if (!(p.tau > 0.5)) return fail(nullptr, CBL_ERR_ARG, "tau must be > 0.5");
  if (!(p.rho0 > 0)) return fail(nullptr, CBL_ERR_ARG, "rho0 must be > 0");
  if (p.prec < CBL_FP64 || p.prec > CBL_FP16DEV) return fail(nullptr, CBL_ERR_ARG, "unknown precision");
  if (!(p.eta > 0) || !(p.rc > 0) || p.nrep < 1 || p.rc > 6.0)
    return fail(nullptr, CBL_ERR_ARG, "eta, rc (<= 6) and nrep must be positive");
  if (alloc && (!alloc->alloc || !alloc->free)) return fail(nullptr, CBL_ERR_ARG, "allocator callbacks missing");
  cbl_ctx* ctx = new cbl_ctx();
  ctx->p = p;
  ctx->ops = lbm_ops(p.q);
  if (alloc) {
    ctx->alloc = *alloc;
    ctx->user_alloc = true;
  }
  if (p.stream) {
    ctx->s = (cudaStream_t)p.stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->s, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return fail(nullptr, CBL_ERR_CUDA, "cudaStreamCreate failed");
    }
    ctx->own_stream = true;
  }
  // the side branch carries the chain of short latency-bound kernels: highest priority, so that
  // their blocks are scheduled ahead of the queued blocks of the bulk collision
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->s);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    for (cudaEvent_t e : {ctx->ev_fork, ctx->ev_join})
      if (e) cudaEventDestroy(e);
    delete ctx;
    return fail(nullptr, CBL_ERR_CUDA, "stream or event creation failed");
  }
  ctx->lat.nx = p.nx;
  ctx->lat.ny = p.ny;
  ctx->lat.nz = p.nz;
  ctx->lat.N = (long long)p.nx * p.ny * p.nz;
  ctx->lat.Ns = pop_stride(ctx->lat.N);
  ctx->prec = (int)p.prec;
  ctx->elem = p.prec == CBL_FP64 ? 8 : (p.prec == CBL_FP32 ? 4 : 2);
  PhysParams& pp = ctx->pp;
  pp.tau = p.tau;
  pp.G = p.G;
  pp.rho0 = p.rho0;
  for (int a = 0; a < 3; ++a) pp.ext[a] = p.ext_force[a];
  pp.eta = p.eta;
  pp.mobility = p.mobility;
  pp.sigma_sf = p.sigma_sf;
  pp.sigma_ss = p.sigma_ss;
  pp.e0 = p.e0;
  pp.rc = p.rc;
  pp.nrep = p.nrep;
  pp.solid_threshold = p.solid_threshold;
  pp.member_threshold = p.member_threshold;
  pp.mpf = p.mpf_kinetics;
  fill_float_params(pp);

  const size_t N = (size_t)ctx->lat.N;
  ctx->fa = dalloc(ctx, (size_t)ctx->lat.Ns * ctx->ops.q * ctx->elem);
  ctx->fb = dalloc(ctx, (size_t)ctx->lat.Ns * ctx->ops.q * ctx->elem);
  // psi of the split and fused passes (the accumulating pass adds a second buffer when chosen)
  ctx->psi = dalloc(ctx, N * (ctx->prec == 0 ? 8 : 4));
  ctx->nbuf = dalloc(ctx, N * 2 * (ctx->prec == 0 ? 8 : 4));
  ctx->flags = (uint16_t*)dalloc(ctx, N * 2);
  ctx->diag_rho = (double*)dalloc(ctx, N * 8);
  ctx->diag_vel = (double*)dalloc(ctx, N * 24);
  ctx->n_mass_part = MASS_SLOTS;
  ctx->mass_part = (double*)dalloc(ctx, (size_t)ctx->n_mass_part * 8);
  ctx->st = (StepState*)dalloc(ctx, sizeof(StepState));
  if (!ctx->fa || !ctx->fb || !ctx->psi || !ctx->nbuf || !ctx->flags || !ctx->diag_rho || !ctx->diag_vel ||
      !ctx->mass_part || !ctx->st) {
    dfree_all(ctx);
    if (ctx->own_stream) cudaStreamDestroy(ctx->s);
    cudaStreamDestroy(ctx->side);
    cudaEventDestroy(ctx->ev_fork);
    cudaEventDestroy(ctx->ev_join);
    delete ctx;
    return fail(nullptr, CBL_ERR_OOM, "device allocation failed");
  }
  cudaMemsetAsync(ctx->flags, 0, N * 2, ctx->s);
  cudaMemsetAsync(ctx->st, 0, sizeof(StepState), ctx->s);
  cudaMemsetAsync(ctx->mass_part, 0, (size_t)ctx->n_mass_part * 8, ctx->s);
  ctx->ops.set_fp16_weights(ctx->s);
  set_repulsion_offsets(p.rc, p.e0, p.nrep, ctx->s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    dfree_all(ctx);
    if (ctx->own_stream) cudaStreamDestroy(ctx->s);
    delete ctx;
    return fail(nullptr, CBL_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e));
  }
  *out = ctx;
  return CBL_OK;
}

cbl_status cbl_add_body(cbl_ctx* ctx, const cbl_body* body, int* body_id) {
  if (!ctx || !body) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  if (ctx->ready) return fail(ctx, CBL_ERR_STATE, "bodies must be added before cbl_init_fluid");
  if ((int)ctx->hb.size() >= MAX_BODIES) return fail(ctx, CBL_ERR_ARG, "too many bodies");
  if (body->shape != 0 && body->shape != 1) return fail(ctx, CBL_ERR_ARG, "shape must be 0 (sphere) or 1 (box)");
  if (!(body->mass_density > 0) || !std::isfinite(body->mass_density))
    return fail(ctx, CBL_ERR_ARG, "mass_density must be finite and > 0");
  if (!(body->wetting_rho >= 0) || !std::isfinite(body->wetting_rho))
    return fail(ctx, CBL_ERR_ARG, "wetting_rho must be finite and >= 0");
  for (int a = 0; a < 3; ++a) {
    // a centre far outside the lattice is almost certainly a mistake, and its tile origin would
    // not fit an int
    if (!(std::fabs(body->center[a]) <= 1e6)) return fail(ctx, CBL_ERR_ARG, "centre must be finite, |c| <= 1e6");
    if (body->shape == 1 && !(body->half[a] > 0 && std::isfinite(body->half[a])))
      return fail(ctx, CBL_ERR_ARG, "box half extents must be finite and > 0");
  }
  for (int a = 0; a < 4; ++a)
    if (!std::isfinite(body->quat[a])) return fail(ctx, CBL_ERR_ARG, "quaternion must be finite");
  if (body->shape == 0 && !(body->radius > 0 && std::isfinite(body->radius)))
    return fail(ctx, CBL_ERR_ARG, "sphere radius must be finite and > 0");
  BodyDev b;
  std::memset(&b, 0, sizeof(b));
  b.shape = body->shape;
  b.radius = body->radius;
  for (int a = 0; a < 3; ++a) {
    b.c0[a] = body->center[a];
    b.half[a] = body->half[a];
    b.X[a] = b.Xprev[a] = body->center[a];
  }
  double qn = std::sqrt(body->quat[0] * body->quat[0] + body->quat[1] * body->quat[1] + body->quat[2] * body->quat[2] +
                        body->quat[3] * body->quat[3]);
  for (int a = 0; a < 4; ++a) b.q0[a] = qn > 0 ? body->quat[a] / qn : (a == 0 ? 1.0 : 0.0);
  for (int a = 0; a < 4; ++a) b.Q[a] = b.q0[a];
  b.rho_s = body->mass_density;
  b.wet = body->wetting_rho;
  b.psi_wet = 1.0 - std::exp(-body->wetting_rho / ctx->p.rho0);
  b.psi_wet_f = (float)b.psi_wet;
  b.fixed = body->fixed;
  // tile: support half-extent + 2 halo layers + half a cell of recentring offset + tile_tail cells
  // (default 2.5) for the discrete profile and the advection tail, which reaches about one cell
  // past R + eta/2 on a body that moved a cell and keeps growing slowly with the distance travelled
  double h[3];
  if (b.shape == 0) {
    for (int a = 0; a < 3; ++a) h[a] = b.radius;
  } else {
    double w = b.q0[0], x = b.q0[1], y = b.q0[2], z = b.q0[3];
    double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                   2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                   2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
    for (int a = 0; a < 3; ++a) h[a] = std::fabs(R[3 * a]) * b.half[0] + std::fabs(R[3 * a + 1]) * b.half[1] +
                                       std::fabs(R[3 * a + 2]) * b.half[2];
  }
  const int n[3] = {ctx->p.nx, ctx->p.ny, ctx->p.nz};
  // a body whose support (surface + eta/2) covers the whole periodic length along an axis is
  // infinite along it (the planar-bridge plates of Sec. 2.1): it turns only about that axis
  b.rot_lock = 0;
  for (int a = 0; a < 3; ++a)
    if (2.0 * (h[a] + 0.5 * ctx->p.eta) >= (double)n[a])
      for (int c = 0; c < 3; ++c)
        if (c != a) b.rot_lock |= 1 << c;
  long long sz = 1;
  for (int a = 0; a < 3; ++a) {
    // sized in double first: a body larger than the lattice takes the whole axis
    const double half = std::ceil(h[a] + 0.5 * ctx->p.eta + 2.5 + ctx->tile_tail);
    int L = 2.0 * half + 1.0 >= (double)n[a] ? n[a] : 2 * (int)half + 1;
    if (L >= n[a]) {
      L = n[a];
      b.o[a] = 0;
    } else {
      b.o[a] = (int)std::floor(b.c0[a] + 0.5) - L / 2;
    }
    b.o_prev[a] = b.o[a];
    b.L[a] = L;
    sz *= L;
  }
  b.sz = sz;
  b.off = ctx->arena_n;
  ctx->arena_n += 3 * sz;
  if (sz > ctx->max_tile) ctx->max_tile = (int)sz;
  ctx->hb.push_back(b);
  if (body_id) *body_id = (int)ctx->hb.size() - 1;
  return CBL_OK;
}

// member boxes to empty before a refill pass outside the step (the step resets them in the body
// kernel); the refill pass rebuilds them
static void reset_member_boxes(cbl_ctx* ctx) { launch_reset_member_boxes(ctx->mbox, (int)ctx->hb.size(), ctx->s); }

// device buffers of the bodies (tables, phase-field arena, per-step sums, boundary list)
static cbl_status alloc_bodies(cbl_ctx* ctx) {
  const int nb = (int)ctx->hb.size();
  if (!nb) return CBL_OK;
  ctx->db = (BodyDev*)dalloc(ctx, sizeof(BodyDev) * nb);
  ctx->arena = (double*)dalloc(ctx, sizeof(double) * (size_t)ctx->arena_n);
  ctx->acc = (double*)dalloc(ctx, sizeof(double) * ACC_N * nb);
  ctx->last = (double*)dalloc(ctx, sizeof(double) * ACC_N * nb);
  ctx->volacc = (double*)dalloc(ctx, sizeof(double) * 2 * nb);
  ctx->fsum = (double*)dalloc(ctx, sizeof(double) * 6 * nb);
  ctx->scratch = (double*)dalloc(ctx, sizeof(double) * 9 * nb);
  for (const BodyDev& b : ctx->hb)
    for (int a = 0; a < 3; ++a) ctx->Lmax = std::max(ctx->Lmax, b.L[a]);
  ctx->rtab = (double*)dalloc(ctx, sizeof(double) * 3 * (size_t)ctx->Lmax * nb);
  ctx->mbox = (int*)dalloc(ctx, sizeof(int) * MBOX_N * nb);
  ctx->blist = (int*)dalloc(ctx, sizeof(int) * (size_t)(ctx->arena_n / 3));
  if (!ctx->db || !ctx->arena || !ctx->acc || !ctx->last || !ctx->volacc || !ctx->fsum || !ctx->scratch || !ctx->blist ||
      !ctx->rtab || !ctx->mbox)
    return fail(ctx, CBL_ERR_OOM, "device allocation failed (bodies)");
  return CBL_OK;
}

// initial density from a liquid mask on the device (NULL mask: vapour everywhere)
__global__ void k_rho_from_mask(double* __restrict__ rho, const unsigned char* __restrict__ mask, long long N,
                                double rho_l, double rho_v) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N) rho[n] = (mask && mask[n]) ? rho_l : rho_v;
}

// rho_host: the initial density field; or, with rho_host NULL, the liquid mask (host, may be NULL)
// and the two densities, expanded on the device
static cbl_status init_common(cbl_ctx* ctx, const double* rho_host, const double* u_host,
                              const unsigned char* mask = nullptr, double rho_l = 0.0, double rho_v = 0.0) {
  const size_t N = (size_t)ctx->lat.N;
  const int nb = (int)ctx->hb.size();
  if (nb) {
    const cbl_status sa = alloc_bodies(ctx);
    if (sa != CBL_OK) return sa;
    for (BodyDev& b : ctx->hb) mirror_f(b);
    CK(cudaMemcpyAsync(ctx->db, ctx->hb.data(), sizeof(BodyDev) * nb, cudaMemcpyHostToDevice, ctx->s));
    CK(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * ACC_N * nb, ctx->s));
    CK(cudaMemsetAsync(ctx->last, 0, sizeof(double) * ACC_N * nb, ctx->s));
    CK(cudaMemsetAsync(ctx->volacc, 0, sizeof(double) * 2 * nb, ctx->s));
    CK(cudaMemsetAsync(ctx->fsum, 0, sizeof(double) * 6 * nb, ctx->s));
    launch_rasterize(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->p.eta, ctx->s);
    launch_neighbour_lists(ctx->db, nb, ctx->lat, ctx->st, ctx->s);
    launch_flags(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->flags, ctx->p.solid_threshold, 1, ctx->st,
                 ctx->s);
    launch_body_props(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->scratch, ctx->s);
  }
  double* drho = (double*)dalloc(ctx, N * 8);
  double* du = u_host ? (double*)dalloc(ctx, N * 24) : nullptr;
  unsigned char* dmask = (!rho_host && mask) ? (unsigned char*)dalloc(ctx, N) : nullptr;
  if (!drho || (u_host && !du) || (!rho_host && mask && !dmask))
    return fail(ctx, CBL_ERR_OOM, "device allocation failed (initial fields)");
  if (rho_host) {
    CK(cudaMemcpyAsync(drho, rho_host, N * 8, cudaMemcpyHostToDevice, ctx->s));
  } else {
    if (dmask) CK(cudaMemcpyAsync(dmask, mask, N, cudaMemcpyHostToDevice, ctx->s));
    k_rho_from_mask<<<(unsigned)((N + 255) / 256), 256, 0, ctx->s>>>(drho, dmask, (long long)N, rho_l, rho_v);
  }
  if (du) CK(cudaMemcpyAsync(du, u_host, N * 24, cudaMemcpyHostToDevice, ctx->s));
  ctx->ops.init_fluid(ctx->prec, ctx->lat, ctx->fa, ctx->flags, drho, du, ctx->s);
  // first boundary-cell list (no cover events yet, so the pass only scans) and member boxes
  reset_member_boxes(ctx);
  ctx->ops.refill(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->db, nb, ctx->max_tile, ctx->st, ctx->blist,
                ctx->arena, ctx->p.member_threshold, ctx->mbox, 0, ctx->s);
  CK(cudaMemsetAsync(ctx->diag_rho, 0, N * 8, ctx->s));
  CK(cudaMemsetAsync(ctx->diag_vel, 0, N * 24, ctx->s));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->s));
  // the initial-field buffers are released right away
  for (void* q : {(void*)drho, (void*)du, (void*)dmask}) {
    if (!q) continue;
    for (size_t k = 0; k < ctx->allocs.size(); ++k)
      if (ctx->allocs[k] == q) {
        if (ctx->user_alloc) ctx->alloc.free(q, ctx->alloc.user);
        else cudaFree(q);
        ctx->allocs.erase(ctx->allocs.begin() + k);
        break;
      }
  }
  ctx->ready = true;
  ctx->psi_valid = false;
  ctx->t = 0;
  return CBL_OK;
}

cbl_status cbl_init_fluid(cbl_ctx* ctx, double rho_liquid, double rho_vapour, const unsigned char* mask) {
  if (!ctx) return fail(ctx, CBL_ERR_ARG, "NULL context");
  if (ctx->ready) return fail(ctx, CBL_ERR_STATE, "already initialised");
  if (!(rho_liquid >= 0) || !(rho_vapour >= 0) || !std::isfinite(rho_liquid) || !std::isfinite(rho_vapour))
    return fail(ctx, CBL_ERR_ARG, "densities must be finite and >= 0");
  return init_common(ctx, nullptr, nullptr, mask, rho_liquid, rho_vapour);
}

cbl_status cbl_init_fluid_fields(cbl_ctx* ctx, const double* rho_host, const double* u_host) {
  if (!ctx || !rho_host) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  if (ctx->ready) return fail(ctx, CBL_ERR_STATE, "already initialised");
  const size_t N = (size_t)ctx->lat.N;
  for (size_t n = 0; n < N; ++n)
    if (!(rho_host[n] >= 0) || !std::isfinite(rho_host[n]))
      return fail(ctx, CBL_ERR_ARG, "initial densities must be finite and >= 0");
  if (u_host)
    for (size_t n = 0; n < 3 * N; ++n)
      if (!std::isfinite(u_host[n])) return fail(ctx, CBL_ERR_ARG, "initial velocities must be finite");
  return init_common(ctx, rho_host, u_host);
}

// phases: 1 density (fused pass: psi over the bodies' tiles only), 2 bulk collision (fused pass:
// with the density), 4 collision of the cells next to a solid
static void enqueue_lbm(cbl_ctx* ctx, int phases, cudaStream_t s) {
  if (ctx->acc_pass) {
    // accumulating pass: phase 1 completes psi of this step (the regions' edge cells, then the bodies'
    // tiles from the populations), phase 2 collides and sums the next step's density
    if (phases & 1) {
      ctx->ops.psi_fixup(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->psi, ctx->psi2, ctx->rhop, ctx->st, ctx->pp,
                         ctx->acc_ty, ctx->acc_sz, s);
      ctx->ops.density_tiles(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->st, ctx->flags, ctx->db, (int)ctx->hb.size(),
                             ctx->max_tile, ctx->psi, ctx->psi2, ctx->pp, s);
    }
    if (phases & 2)
      ctx->ops.lbm_acc(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->psi, ctx->psi2, ctx->rhop, ctx->db,
                       ctx->mass_part, ctx->st, ctx->diag_rho, ctx->diag_vel, ctx->pp, ctx->acc_ty, ctx->acc_sz, s);
    if (phases & 4)
      ctx->ops.lbm_step(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->psi, ctx->psi2, ctx->db,
                        ctx->mass_part, (unsigned)ctx->block_x, ctx->st, ctx->diag_rho, ctx->diag_vel, ctx->pp,
                        ctx->nbuf, ctx->blist, s, 4);
    return;
  }
  if (ctx->fused_tz) {
    if (phases & 1)
      ctx->ops.density_tiles(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->st, ctx->flags, ctx->db, (int)ctx->hb.size(),
                             ctx->max_tile, ctx->psi, nullptr, ctx->pp, s);
    if (phases & 2)
      ctx->ops.lbm_fused(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->db, ctx->mass_part, ctx->st,
                         ctx->diag_rho, ctx->diag_vel, ctx->pp, ctx->fused_tz, ctx->fused_ty, s);
    if (phases & 4)
      ctx->ops.lbm_step(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->psi, nullptr, ctx->db,
                        ctx->mass_part, (unsigned)ctx->block_x, ctx->st, ctx->diag_rho, ctx->diag_vel, ctx->pp,
                        ctx->nbuf, ctx->blist, s, 4);
  } else {
    ctx->ops.lbm_step(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->psi, nullptr, ctx->db, ctx->mass_part,
                    (unsigned)ctx->block_x, ctx->st, ctx->diag_rho, ctx->diag_vel, ctx->pp, ctx->nbuf, ctx->blist,
                    s, phases);
  }
}

static const int KEV_RING = 512;

// bulk collision, bracketed by the timing events when "kernel_events" is on
static void enqueue_bulk(cbl_ctx* ctx, cudaStream_t s) {
  if (ctx->kev) cudaEventRecordWithFlags(ctx->kev_cap[0], s, cudaEventRecordExternal);
  enqueue_lbm(ctx, 2, s);
  if (ctx->kev) cudaEventRecordWithFlags(ctx->kev_cap[1], s, cudaEventRecordExternal);
}

// One step, enqueued for capture into a graph. With bodies, the collision of the cells next to a
// solid, the solid-fluid force pass and the solid-solid repulsion run on a side branch beside the
// bulk collision (they touch other cells, or only the phase fields, and add into the force
// accumulators with atomics); the body update joins both.
static void enqueue_step(cbl_ctx* ctx) {
  const int nb = (int)ctx->hb.size();
  auto phase_update = [&](cudaStream_t s) {
    launch_advect(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->pp.mpf, ctx->volacc, ctx->st, ctx->rtab,
                  ctx->Lmax, s);
    if (ctx->pp.mpf) launch_kinetics(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->volacc, ctx->pp, s);
  };
  auto flags_refill = [&](cudaStream_t s) {
    launch_flags(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->flags, ctx->p.solid_threshold, 0, ctx->st,
                 s);
    ctx->ops.refill(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->db, nb, ctx->max_tile, ctx->st, ctx->blist,
                  ctx->arena, ctx->p.member_threshold, ctx->mbox, 1, s);
  };
  if (nb && ctx->branches) {
    // The bulk collision (every cell without a solid neighbour) runs beside the chain that needs only
    // the source populations, psi and the phase fields: collision of the cells next to a solid, force
    // pass, repulsion, body update, advection, kinetics. That chain is the longer path and is made
    // of small latency-bound kernels, so it runs on the high-priority side stream, whose blocks are
    // scheduled ahead of the bulk collision's queued ones. The flag update and the refill rewrite
    // what the bulk collision reads and writes, so they wait for both. With the fused pass, psi of the
    // bodies' tiles (all that the side chain needs) is the side chain's first kernel.
    if (!ctx->fused_tz) enqueue_lbm(ctx, 1, ctx->s);
    cudaEventRecord(ctx->ev_fork, ctx->s);
    cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
    if (ctx->fused_tz) enqueue_lbm(ctx, 1, ctx->side);
    enqueue_lbm(ctx, 4, ctx->side);
    ctx->ops.boundary(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->db, nb, ctx->acc, ctx->blist, ctx->st,
                    ctx->nbuf, ctx->pp.G, ctx->side);
    launch_repulsion(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->acc, ctx->pp, ctx->mbox, ctx->side);
    launch_bodies(ctx->lat, ctx->db, nb, ctx->acc, ctx->last, ctx->volacc, ctx->st, ctx->rtab, ctx->Lmax, ctx->mbox, ctx->fsum,
                  ctx->side);
    phase_update(ctx->side);
    cudaEventRecord(ctx->ev_join, ctx->side);
    enqueue_bulk(ctx, ctx->s);
    cudaStreamWaitEvent(ctx->s, ctx->ev_join, 0);
    flags_refill(ctx->s);
  } else {
    enqueue_lbm(ctx, 1, ctx->s);
    enqueue_bulk(ctx, ctx->s);
    enqueue_lbm(ctx, 4, ctx->s);
    ctx->ops.boundary(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->db, nb, ctx->acc, ctx->blist, ctx->st,
                    ctx->nbuf, ctx->pp.G, ctx->s);
    if (nb) {
      launch_repulsion(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->acc, ctx->pp, ctx->mbox, ctx->s);
      launch_bodies(ctx->lat, ctx->db, nb, ctx->acc, ctx->last, ctx->volacc, ctx->st, ctx->rtab, ctx->Lmax,
                    ctx->mbox, ctx->fsum, ctx->s);
      phase_update(ctx->s);
      flags_refill(ctx->s);
    }
  }
  launch_finish(ctx->mass_part, ctx->n_mass_part, ctx->st, ctx->s);
}

// The part of a step that follows the bulk lattice-Boltzmann pass in a persistent batch launch: the
// collision of the cells next to a solid, the bodies' chain, flags and refill, the step's end.
static void enqueue_side_chain(cbl_ctx* ctx) {
  const int nb = (int)ctx->hb.size();
  enqueue_lbm(ctx, 4, ctx->s);
  if (nb) {
    ctx->ops.boundary(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->db, nb, ctx->acc, ctx->blist, ctx->st,
                      ctx->nbuf, ctx->pp.G, ctx->s);
    launch_repulsion(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->acc, ctx->pp, ctx->mbox, ctx->s);
    launch_bodies(ctx->lat, ctx->db, nb, ctx->acc, ctx->last, ctx->volacc, ctx->st, ctx->rtab, ctx->Lmax, ctx->mbox, ctx->fsum,
                  ctx->s);
    launch_advect(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->pp.mpf, ctx->volacc, ctx->st, ctx->rtab,
                  ctx->Lmax, ctx->s);
    if (ctx->pp.mpf) launch_kinetics(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->volacc, ctx->pp, ctx->s);
    launch_flags(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->flags, ctx->p.solid_threshold, 0, ctx->st,
                 ctx->s);
    ctx->ops.refill(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->db, nb, ctx->max_tile, ctx->st, ctx->blist,
                    ctx->arena, ctx->p.member_threshold, ctx->mbox, 1, ctx->s);
  }
  launch_finish(ctx->mass_part, ctx->n_mass_part, ctx->st, ctx->s);
}

// Accumulating pass: its buffers, its kernel's shared-memory limit, its region depth, and psi of
// the current step, which the pass computes in the step before. psi is not in place after
// initialisation, a checkpoint load, a move of the bodies, an option change, kernel-by-kernel timing
// or a batch step: then a whole-lattice density pass computes it, and StepState::psi_skip tells the
// fix-up and the tile pass of the next step to leave it as it is.
static cbl_status acc_prepare(cbl_ctx* ctx) {
  if (!ctx->acc_pass) return CBL_OK;
  const size_t N = (size_t)ctx->lat.N, el = ctx->prec == 0 ? 8 : 4;
  if (!ctx->psi2) ctx->psi2 = dalloc(ctx, N * el);
  if (!ctx->rhop) ctx->rhop = dalloc(ctx, N * el);
  if (!ctx->psi2 || !ctx->rhop) return fail(ctx, CBL_ERR_OOM, "device allocation failed (accumulating pass)");
  ctx->acc_sz = ctx->acc_sz_req > 0 ? ctx->acc_sz_req : ctx->ops.acc_sz(ctx->lat, ctx->prec, ctx->acc_ty, 2);
  if (ctx->acc_attr_ty != ctx->acc_ty) {
    // a zero-plane call outside any capture sets the kernel's dynamic shared-memory limit
    Lat none = ctx->lat;
    none.nz = 0;
    CK(ctx->ops.lbm_acc(ctx->prec, none, ctx->fa, ctx->fb, ctx->flags, ctx->psi, ctx->psi2, ctx->rhop, ctx->db,
                        ctx->mass_part, ctx->st, ctx->diag_rho, ctx->diag_vel, ctx->pp, ctx->acc_ty, 1, ctx->s));
    ctx->acc_attr_ty = ctx->acc_ty;
  }
  if (!ctx->psi_valid) {
    ctx->ops.lbm_step(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->psi, ctx->psi2, ctx->db, ctx->mass_part,
                      (unsigned)ctx->block_x, ctx->st, ctx->diag_rho, ctx->diag_vel, ctx->pp, ctx->nbuf, ctx->blist,
                      ctx->s, 1);
    CK(cudaMemsetAsync(&ctx->st->psi_skip, 1, 1, ctx->s));
    CK(cudaGetLastError());
    ctx->psi_valid = true;
  }
  return CBL_OK;
}

cbl_status cbl_step(cbl_ctx* ctx, int nsteps) {
  if (!ctx) return fail(ctx, CBL_ERR_ARG, "NULL context");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "cbl_step before cbl_init_fluid");
  if (nsteps < 0) return fail(ctx, CBL_ERR_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return CBL_OK;
  {
    const cbl_status sa = acc_prepare(ctx);
    if (sa != CBL_OK) return sa;
  }
  if (!ctx->gexec) {
    CK(cudaStreamBeginCapture(ctx->s, cudaStreamCaptureModeThreadLocal));
    enqueue_step(ctx);
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamEndCapture(ctx->s, &ctx->graph);
    CK(e1);
    CK(e2);
    // the side stream's priority is recorded on its kernel nodes; the executable graph honours it
    // only with this flag
    CK(cudaGraphInstantiate(&ctx->gexec, ctx->graph, ctx->node_priority ? cudaGraphInstantiateFlagUseNodePriority : 0));
    if (ctx->kev) {
      // the two event-record nodes that bracket the bulk collision
      size_t nn = 0;
      CK(cudaGraphGetNodes(ctx->graph, nullptr, &nn));
      std::vector<cudaGraphNode_t> nodes(nn);
      CK(cudaGraphGetNodes(ctx->graph, nodes.data(), &nn));
      ctx->kev_node[0] = ctx->kev_node[1] = nullptr;
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        CK(cudaGraphNodeGetType(nd, &ty));
        if (ty != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        for (int k = 0; k < 2; ++k)
          if (ev == ctx->kev_cap[k]) ctx->kev_node[k] = nd;
      }
      if (!ctx->kev_node[0] || !ctx->kev_node[1])
        return fail(ctx, CBL_ERR_CUDA, "timing events of the bulk collision not found in the step graph");
    }
  }
  // the diag word is tested for non-zero: byte-wise memsets keep the whole call asynchronous
  CK(cudaMemsetAsync(&ctx->st->diag, 0, sizeof(int), ctx->s));
  for (int k = 0; k < nsteps; ++k) {
    if (k == nsteps - 1) CK(cudaMemsetAsync(&ctx->st->diag, 1, sizeof(int), ctx->s));
    if (ctx->kev) {
      const int r = k % KEV_RING;
      CK(cudaGraphExecEventRecordNodeSetEvent(ctx->gexec, ctx->kev_node[0], ctx->kev_ring[2 * r]));
      CK(cudaGraphExecEventRecordNodeSetEvent(ctx->gexec, ctx->kev_node[1], ctx->kev_ring[2 * r + 1]));
    }
    CK(cudaGraphLaunch(ctx->gexec, ctx->s));
  }
  ctx->kev_steps = nsteps;
  ctx->t += nsteps;
  ctx->fsum_steps += nsteps;
  return CBL_OK;
}

cbl_status cbl_kernel_times(cbl_ctx* ctx, int max, float* ms, int* count) {
  if (!ctx || !ms || !count || max < 0) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  if (!ctx->kev) return fail(ctx, CBL_ERR_STATE, "option kernel_events is off");
  CK(cudaStreamSynchronize(ctx->s));
  const long long have = std::min<long long>(ctx->kev_steps, KEV_RING);
  const int n = (int)std::min<long long>(have, (long long)max);
  // the last n replays, oldest first
  for (int j = 0; j < n; ++j) {
    const long long k = ctx->kev_steps - n + j;
    const int r = (int)(k % KEV_RING);
    CK(cudaEventElapsedTime(&ms[j], ctx->kev_ring[2 * r], ctx->kev_ring[2 * r + 1]));
  }
  *count = n;
  return CBL_OK;
}

cbl_status cbl_time_phases(cbl_ctx* ctx, int nsteps, double* ms) {
  if (!ctx || !ms) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "cbl_time_phases before cbl_init_fluid");
  if (nsteps <= 0) return fail(ctx, CBL_ERR_ARG, "nsteps must be > 0");
  const int nb = (int)ctx->hb.size();
  cudaEvent_t ev[CBL_NPHASES + 1];
  for (int k = 0; k <= CBL_NPHASES; ++k) CK(cudaEventCreate(&ev[k]));
  double acc[CBL_NPHASES] = {0};
  {
    const cbl_status sa = acc_prepare(ctx);
    if (sa != CBL_OK) return sa;
  }
  CK(cudaMemsetAsync(&ctx->st->diag, 0, sizeof(int), ctx->s));
  for (int it = 0; it < nsteps; ++it) {
    CK(cudaEventRecord(ev[0], ctx->s));
    enqueue_lbm(ctx, 1, ctx->s);
    CK(cudaEventRecord(ev[1], ctx->s));
    enqueue_lbm(ctx, 6, ctx->s);
    CK(cudaEventRecord(ev[2], ctx->s));
    ctx->ops.boundary(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->db, nb, ctx->acc, ctx->blist, ctx->st,
                    ctx->nbuf, ctx->pp.G, ctx->s);
    CK(cudaEventRecord(ev[3], ctx->s));
    if (nb) launch_repulsion(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->acc, ctx->pp, ctx->mbox, ctx->s);
    CK(cudaEventRecord(ev[4], ctx->s));
    launch_bodies(ctx->lat, ctx->db, nb, ctx->acc, ctx->last, ctx->volacc, ctx->st, ctx->rtab, ctx->Lmax, ctx->mbox, ctx->fsum,
                  ctx->s);
    CK(cudaEventRecord(ev[5], ctx->s));
    if (nb)
      launch_advect(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->pp.mpf, ctx->volacc, ctx->st, ctx->rtab,
                    ctx->Lmax, ctx->s);
    CK(cudaEventRecord(ev[6], ctx->s));
    if (nb && ctx->pp.mpf)
      launch_kinetics(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->volacc, ctx->pp, ctx->s);
    CK(cudaEventRecord(ev[7], ctx->s));
    if (nb)
      launch_flags(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->flags, ctx->p.solid_threshold, 0, ctx->st,
                   ctx->s);
    CK(cudaEventRecord(ev[8], ctx->s));
    if (nb)
      ctx->ops.refill(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->db, nb, ctx->max_tile, ctx->st, ctx->blist,
                    ctx->arena, ctx->p.member_threshold, ctx->mbox, 1, ctx->s);
    launch_finish(ctx->mass_part, ctx->n_mass_part, ctx->st, ctx->s);
    CK(cudaEventRecord(ev[9], ctx->s));
    CK(cudaGetLastError());
    CK(cudaEventSynchronize(ev[9]));
    for (int k = 0; k < CBL_NPHASES; ++k) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
      acc[k] += t;
    }
  }
  for (int k = 0; k <= CBL_NPHASES; ++k) cudaEventDestroy(ev[k]);
  for (int k = 0; k < CBL_NPHASES; ++k) ms[k] = acc[k] / nsteps;
  ctx->psi_valid = false;  // these steps computed psi at their start, not for the step after
  ctx->t += nsteps;
  ctx->fsum_steps += nsteps;
  return CBL_OK;
}

cbl_status cbl_read_fields(cbl_ctx* ctx, double* rho, double* vel, double* phi_fluid, int on_device) {
  if (!ctx) return fail(ctx, CBL_ERR_ARG, "NULL context");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "not initialised");
  const size_t N = (size_t)ctx->lat.N;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaStreamSynchronize(ctx->s));
  if (rho) CK(cudaMemcpyAsync(rho, ctx->diag_rho, N * 8, k, ctx->s));
  if (vel) CK(cudaMemcpyAsync(vel, ctx->diag_vel, N * 24, k, ctx->s));
  if (phi_fluid) {
    if (!ctx->dense && !(ctx->dense = (double*)dalloc(ctx, N * 8))) return fail(ctx, CBL_ERR_OOM, "dense buffer");
    launch_phi_dense(ctx->lat, ctx->db, (int)ctx->hb.size(), ctx->max_tile, ctx->arena, -1, ctx->dense, ctx->s);
    CK(cudaMemcpyAsync(phi_fluid, ctx->dense, N * 8, k, ctx->s));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->s));
  return CBL_OK;
}

cbl_status cbl_velocity_set(cbl_ctx* ctx, int* q, int* c, double* w) {
  if (!ctx) return fail(ctx, CBL_ERR_ARG, "NULL context");
  const int Qn = ctx->ops.q;
  if (q) *q = Qn;
  for (int i = 0; i < Qn; ++i) {
    if (c) {
      c[3 * i] = Qn == 27 ? q27::cx_of(i) : q19::cx_of(i);
      c[3 * i + 1] = Qn == 27 ? q27::cy_of(i) : q19::cy_of(i);
      c[3 * i + 2] = Qn == 27 ? q27::cz_of(i) : q19::cz_of(i);
    }
    if (w) w[i] = Qn == 27 ? q27::w_of(i) : q19::w_of(i);
  }
  return CBL_OK;
}

cbl_status cbl_read_populations(cbl_ctx* ctx, double* out, int on_device) {
  if (!ctx || !out) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "not initialised");
  const size_t bytes = (size_t)ctx->ops.q * ctx->lat.N * 8;
  double* dst = out;
  if (!on_device) {
    if (!ctx->popbuf && !(ctx->popbuf = (double*)dalloc(ctx, bytes))) return fail(ctx, CBL_ERR_OOM, "population buffer");
    dst = ctx->popbuf;
  }
  ctx->ops.read_populations(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->st, ctx->flags, dst, ctx->s);
  CK(cudaGetLastError());
  if (!on_device) CK(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  return CBL_OK;
}

cbl_status cbl_read_flags(cbl_ctx* ctx, unsigned char* solid, int32_t* owner) {
  if (!ctx) return fail(ctx, CBL_ERR_ARG, "NULL context");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "not initialised");
  std::vector<uint16_t> f((size_t)ctx->lat.N);
  CK(cudaMemcpyAsync(f.data(), ctx->flags, f.size() * 2, cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  for (size_t n = 0; n < f.size(); ++n) {
    bool s = f[n] & F_SOLID;
    if (solid) solid[n] = s ? 1 : 0;
    if (owner) owner[n] = s ? (int32_t)(f[n] & F_OWNER) : -1;
  }
  return CBL_OK;
}

cbl_status cbl_read_phi(cbl_ctx* ctx, int body, double* phi_host) {
  if (!ctx || !phi_host) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "not initialised");
  if (body < 0 || body >= (int)ctx->hb.size()) return fail(ctx, CBL_ERR_ARG, "body id out of range");
  const size_t N = (size_t)ctx->lat.N;
  if (!ctx->dense && !(ctx->dense = (double*)dalloc(ctx, N * 8))) return fail(ctx, CBL_ERR_OOM, "dense buffer");
  launch_phi_dense(ctx->lat, ctx->db, (int)ctx->hb.size(), ctx->max_tile, ctx->arena, body, ctx->dense, ctx->s);
  CK(cudaMemcpyAsync(phi_host, ctx->dense, N * 8, cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->s));
  return CBL_OK;
}

cbl_status cbl_read_body_forces(cbl_ctx* ctx, double* F, double* T, double* parts) {
  if (!ctx) return fail(ctx, CBL_ERR_ARG, "NULL context");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "not initialised");
  const int nb = (int)ctx->hb.size();
  if (!nb) return CBL_OK;
  std::vector<double> h((size_t)nb * ACC_N);
  CK(cudaMemcpyAsync(h.data(), ctx->last, h.size() * 8, cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  for (int b = 0; b < nb; ++b) {
    const double* a = &h[(size_t)b * ACC_N];
    for (int k = 0; k < 3; ++k) {
      if (F) F[3 * b + k] = a[ACC_MOM_F + k] + a[ACC_ADH_F + k] + a[ACC_REP_F + k];
      if (T) T[3 * b + k] = a[ACC_MOM_T + k] + a[ACC_ADH_T + k] + a[ACC_REP_T + k];
    }
    if (parts)
      for (int k = 0; k < ACC_N; ++k) parts[(size_t)b * ACC_N + k] = a[k];
  }
  return CBL_OK;
}

// CBL_ERR_UNSTABLE once a body update was not finite (device error bit E_UNSTABLE; that body is
// held at its last finite pose)
static cbl_status unstable_check(cbl_ctx* ctx) {
  StepState h;
  CK(cudaMemcpyAsync(&h, ctx->st, sizeof(h), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  if (h.err & E_UNSTABLE) return fail(ctx, CBL_ERR_UNSTABLE, "a body update was not finite; the body is held");
  return CBL_OK;
}

cbl_status cbl_read_force_mean(cbl_ctx* ctx, double* F, double* T, long long* nsteps, int reset) {
  if (!ctx) return fail(ctx, CBL_ERR_ARG, "NULL context");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "not initialised");
  const int nb = (int)ctx->hb.size();
  if (nsteps) *nsteps = ctx->fsum_steps;
  if (!nb) return CBL_OK;
  std::vector<double> h((size_t)6 * nb);
  CK(cudaMemcpyAsync(h.data(), ctx->fsum, h.size() * 8, cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  const double inv = ctx->fsum_steps ? 1.0 / (double)ctx->fsum_steps : 0.0;
  for (int b = 0; b < nb; ++b)
    for (int c = 0; c < 3; ++c) {
      if (F) F[3 * b + c] = h[6 * b + c] * inv;
      if (T) T[3 * b + c] = h[6 * b + 3 + c] * inv;
    }
  if (reset) {
    CK(cudaMemsetAsync(ctx->fsum, 0, sizeof(double) * 6 * nb, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    ctx->fsum_steps = 0;
  }
  return CBL_OK;
}

cbl_status cbl_get_bodies(cbl_ctx* ctx, double* X, double* V, double* W, double* Qo, double* M, double* I) {
  if (!ctx) return fail(ctx, CBL_ERR_ARG, "NULL context");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "not initialised");
  const int nb = (int)ctx->hb.size();
  if (!nb) return CBL_OK;
  std::vector<BodyDev> h(nb);
  CK(cudaMemcpyAsync(h.data(), ctx->db, sizeof(BodyDev) * nb, cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  for (int b = 0; b < nb; ++b) {
    for (int a = 0; a < 3; ++a) {
      if (X) X[3 * b + a] = h[b].X[a];
      if (V) V[3 * b + a] = h[b].V[a];
      if (W) W[3 * b + a] = h[b].W[a];
    }
    if (Qo)
      for (int a = 0; a < 4; ++a) Qo[4 * b + a] = h[b].Q[a];
    if (M) M[b] = h[b].M;
    if (I)
      for (int a = 0; a < 9; ++a) I[9 * b + a] = h[b].Ib[a];
  }
  return unstable_check(ctx);
}

cbl_status cbl_move_bodies(cbl_ctx* ctx, const double* X, const double* Qn, const double* V, const double* W) {
  if (!ctx || !X) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "not initialised");
  const int nb = (int)ctx->hb.size();
  if (!nb) return CBL_OK;
  for (int k = 0; k < 3 * nb; ++k)
    if ((V && !std::isfinite(V[k])) || (W && !std::isfinite(W[k])))
      return fail(ctx, CBL_ERR_ARG, "velocities must be finite");
  ctx->psi_valid = false;  // flags and populations change
  std::vector<BodyDev> h0(nb), h(nb);
  CK(cudaMemcpyAsync(h0.data(), ctx->db, sizeof(BodyDev) * nb, cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  const int n[3] = {ctx->p.nx, ctx->p.ny, ctx->p.nz};
  // target poses, and the largest displacement of a body surface point (translation plus rotation
  // angle times the body's extent; a sphere's rotation does not move its phase field)
  std::vector<double> Xt(3 * nb), Qt(4 * nb);
  double disp = 0.0;
  for (int b = 0; b < nb; ++b) {
    const BodyDev& d = h0[b];
    double dx2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      if (!std::isfinite(X[3 * b + a])) return fail(ctx, CBL_ERR_ARG, "non-finite body position");
      double x = std::fmod(X[3 * b + a], (double)n[a]);
      if (x < 0) x += n[a];
      Xt[3 * b + a] = x;
      const double dd = mimg(x - d.X[a], n[a]);
      dx2 += dd * dd;
    }
    double dot = 0.0;
    if (Qn) {
      const double* q = Qn + 4 * b;
      const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
      if (!(qn > 0) || !std::isfinite(qn)) return fail(ctx, CBL_ERR_ARG, "zero or non-finite quaternion");
      for (int a = 0; a < 4; ++a) {
        Qt[4 * b + a] = q[a] / qn;
        dot += Qt[4 * b + a] * d.Q[a];
      }
    } else {
      for (int a = 0; a < 4; ++a) Qt[4 * b + a] = d.Q[a];
      dot = 1.0;
    }
    const double ext = d.shape == 0 ? 0.0 : std::sqrt(d.half[0] * d.half[0] + d.half[1] * d.half[1] + d.half[2] * d.half[2]);
    const double ang = 2.0 * std::acos(std::min(1.0, std::fabs(dot)));
    disp = std::max(disp, std::sqrt(dx2) + ang * ext);
  }
  // a move of at most half a cell per sub-move keeps a fluid node next to every newly covered one,
  // so each cover refill finds a receiver
  const int nsub = (int)std::min(4096.0, std::max(1.0, std::ceil(disp / 0.5)));
  for (int k = 1; k <= nsub; ++k) {
    const double s = (double)k / nsub;
    for (int b = 0; b < nb; ++b) {
      BodyDev d = h0[b];
      for (int a = 0; a < 3; ++a) {
        double x = k == nsub ? Xt[3 * b + a] : d.X[a] + s * mimg(Xt[3 * b + a] - d.X[a], n[a]);
        x = std::fmod(x, (double)n[a]);
        if (x < 0) x += n[a];
        d.X[a] = d.Xprev[a] = d.c0[a] = x;
      }
      // normalised linear blend of the quaternions, taken along the shorter arc
      double q[4], sgn = 0.0, qn = 0.0;
      for (int a = 0; a < 4; ++a) sgn += h0[b].Q[a] * Qt[4 * b + a];
      sgn = sgn < 0 ? -1.0 : 1.0;
      for (int a = 0; a < 4; ++a) {
        q[a] = k == nsub ? Qt[4 * b + a] : (1.0 - s) * h0[b].Q[a] + s * sgn * Qt[4 * b + a];
        qn += q[a] * q[a];
      }
      qn = std::sqrt(qn);
      for (int a = 0; a < 4; ++a) d.Q[a] = d.q0[a] = q[a] / qn;
      if (k == nsub) {
        for (int a = 0; a < 3; ++a) {
          if (V) d.V[a] = V[3 * b + a];
          if (W) d.W[a] = W[3 * b + a];
        }
      }
      for (int a = 0; a < 3; ++a) {
        if (d.L[a] < n[a]) d.o[a] = (int)std::floor(d.X[a] + 0.5) - d.L[a] / 2;
        d.o_prev[a] = d.o[a];
      }
      h[b] = d;
    }
    // solid cells hand nothing over (a node covered by the last pass still holds its populations,
    // already given to its neighbours): zero them, then clear the flags under the current tiles
    ctx->ops.zero_solid(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->st, ctx->flags, ctx->db, nb, ctx->max_tile, ctx->s);
    launch_clear_tile_flags(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->flags, ctx->s);
    for (BodyDev& b : h) mirror_f(b);
    CK(cudaMemcpyAsync(ctx->db, h.data(), sizeof(BodyDev) * nb, cudaMemcpyHostToDevice, ctx->s));
    launch_rasterize(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->p.eta, ctx->s);
    launch_neighbour_lists(ctx->db, nb, ctx->lat, ctx->st, ctx->s);
    // cover events are counted by the flag pass; the boundary list is rebuilt by the refill pass
    CK(cudaMemsetAsync(&ctx->st->ncover, 0, sizeof(unsigned), ctx->s));
    CK(cudaMemsetAsync(&ctx->st->nbnd, 0, sizeof(unsigned), ctx->s));
    launch_flags(ctx->lat, ctx->db, nb, ctx->max_tile, ctx->arena, ctx->flags, ctx->p.solid_threshold, 0, ctx->st,
                 ctx->s);
    launch_clear_stale(ctx->lat, ctx->flags, ctx->s);
    reset_member_boxes(ctx);
    ctx->ops.refill(ctx->prec, ctx->lat, ctx->fa, ctx->fb, ctx->flags, ctx->db, nb, ctx->max_tile, ctx->st, ctx->blist,
                  ctx->arena, ctx->p.member_threshold, ctx->mbox, 0, ctx->s);
    CK(cudaGetLastError());
    // the host copy h (and the device memcpy source) must outlive the copy
    CK(cudaStreamSynchronize(ctx->s));
  }
  return CBL_OK;
}

cbl_status cbl_set_body_velocities(cbl_ctx* ctx, const double* V, const double* W) {
  if (!ctx) return fail(ctx, CBL_ERR_ARG, "NULL context");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "not initialised");
  const int nb = (int)ctx->hb.size();
  if (!nb) return CBL_OK;
  for (int k = 0; k < 3 * nb; ++k)
    if ((V && !std::isfinite(V[k])) || (W && !std::isfinite(W[k])))
      return fail(ctx, CBL_ERR_ARG, "velocities must be finite");
  std::vector<BodyDev> h(nb);
  CK(cudaMemcpyAsync(h.data(), ctx->db, sizeof(BodyDev) * nb, cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  for (int b = 0; b < nb; ++b)
    for (int a = 0; a < 3; ++a) {
      if (V) h[b].V[a] = V[3 * b + a];
      if (W) h[b].W[a] = W[3 * b + a];
    }
  for (BodyDev& b : h) mirror_f(b);
  CK(cudaMemcpyAsync(ctx->db, h.data(), sizeof(BodyDev) * nb, cudaMemcpyHostToDevice, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  return CBL_OK;
}

cbl_status cbl_set_bodies_fixed(cbl_ctx* ctx, const int* fixed) {
  if (!ctx || !fixed) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "not initialised");
  const int nb = (int)ctx->hb.size();
  if (!nb) return CBL_OK;
  std::vector<BodyDev> h(nb);
  CK(cudaMemcpyAsync(h.data(), ctx->db, sizeof(BodyDev) * nb, cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  for (int b = 0; b < nb; ++b) {
    h[b].fixed = ctx->hb[b].fixed = fixed[b] ? 1 : 0;
    if (h[b].fixed)
      for (int a = 0; a < 3; ++a) h[b].V[a] = h[b].W[a] = 0.0;
    mirror_f(h[b]);
  }
  CK(cudaMemcpyAsync(ctx->db, h.data(), sizeof(BodyDev) * nb, cudaMemcpyHostToDevice, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  return CBL_OK;
}

// ---- checkpoint / resume -------------------------------------------------------------------------
// File: magic, version, the parameters that shape the state, the host scalars, then every device
// buffer that carries state from one step to the next (both population buffers, flags, the last
// step's fields, the body table, phase-field arena, force sums, boundary list, step state). The
// scratch that each step rebuilds (psi, the near-solid side buffer, mass partials, offset tables)
// is not stored.
static const char CKPT_MAGIC[8] = {'C', 'B', 'L', 'S', 'T', 'A', 'T', 'E'};
static const int CKPT_VERSION = 2;

namespace {
struct CkptHeader {
  char magic[8];
  int version, q, prec, nb;
  int nx, ny, nz, Lmax;
  long long N, Ns, arena_n, t;
  double tau, G, rho0, ext[3], mobility, eta, sigma_sf, sigma_ss, e0, rc, solid_thr, member_thr;
  int mpf, nrep;
};
// the header is compared with memcmp after a struct copy, which need not keep padding bytes: the
// members are laid out so that there are none
static_assert(sizeof(CkptHeader) == 8 + 8 * sizeof(int) + 4 * sizeof(long long) + 14 * sizeof(double) +
                                        2 * sizeof(int),
              "CkptHeader must have no implicit padding");

struct Buf {
  void* dev;
  size_t bytes;
};
}  // namespace

static CkptHeader ckpt_header(const cbl_ctx* ctx) {
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, CKPT_MAGIC, 8);
  h.version = CKPT_VERSION;
  h.q = ctx->ops.q;
  h.prec = ctx->prec;
  h.nb = (int)ctx->hb.size();
  h.nx = ctx->p.nx;
  h.ny = ctx->p.ny;
  h.nz = ctx->p.nz;
  h.Lmax = ctx->Lmax;
  h.N = ctx->lat.N;
  h.Ns = ctx->lat.Ns;
  h.arena_n = ctx->arena_n;
  h.t = ctx->t;
  h.tau = ctx->p.tau;
  h.G = ctx->p.G;
  h.rho0 = ctx->p.rho0;
  for (int a = 0; a < 3; ++a) h.ext[a] = ctx->p.ext_force[a];
  h.mobility = ctx->p.mobility;
  h.eta = ctx->p.eta;
  h.sigma_sf = ctx->p.sigma_sf;
  h.sigma_ss = ctx->p.sigma_ss;
  h.e0 = ctx->p.e0;
  h.rc = ctx->p.rc;
  h.solid_thr = ctx->p.solid_threshold;
  h.member_thr = ctx->p.member_threshold;
  h.mpf = ctx->p.mpf_kinetics;
  h.nrep = ctx->p.nrep;
  return h;
}

static std::vector<Buf> ckpt_buffers(cbl_ctx* ctx) {
  const size_t N = (size_t)ctx->lat.N, nb = ctx->hb.size();
  const size_t pop = (size_t)ctx->lat.Ns * ctx->ops.q * ctx->elem;
  std::vector<Buf> v = {{ctx->fa, pop},       {ctx->fb, pop},           {ctx->flags, N * 2},
                        {ctx->diag_rho, N * 8}, {ctx->diag_vel, N * 24}, {ctx->st, sizeof(StepState)}};
  if (nb) {
    v.push_back({ctx->arena, sizeof(double) * (size_t)ctx->arena_n});
    v.push_back({ctx->acc, sizeof(double) * ACC_N * nb});
    v.push_back({ctx->last, sizeof(double) * ACC_N * nb});
    v.push_back({ctx->volacc, sizeof(double) * 2 * nb});
    v.push_back({ctx->mbox, sizeof(int) * MBOX_N * nb});
    v.push_back({ctx->blist, sizeof(int) * (size_t)(ctx->arena_n / 3)});
  }
  return v;
}

// a copy ordered on the context's stream (its buffers come from a stream-ordered allocator), waited for
static cbl_status copy_sync(cbl_ctx* ctx, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
  cbl_status st = cuda_check(ctx, cudaMemcpyAsync(dst, src, bytes, kind, ctx->s), "checkpoint copy");
  if (st == CBL_OK) st = cuda_check(ctx, cudaStreamSynchronize(ctx->s), "checkpoint copy");
  return st;
}

cbl_status cbl_save(cbl_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "cbl_save before cbl_init_fluid");
  CK(cudaStreamSynchronize(ctx->s));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(ctx, CBL_ERR_ARG, std::string("cannot open ") + path + " for writing");
  const CkptHeader h = ckpt_header(ctx);
  bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
  const int nb = (int)ctx->hb.size();
  std::vector<BodyDev> bodies(nb);
  cbl_status st = CBL_OK;
  if (nb) {
    st = copy_sync(ctx, bodies.data(), ctx->db, sizeof(BodyDev) * nb, cudaMemcpyDeviceToHost);
    ok = ok && st == CBL_OK && std::fwrite(bodies.data(), sizeof(BodyDev), nb, f) == (size_t)nb;
  }
  std::vector<char> host;
  for (const Buf& b : ckpt_buffers(ctx)) {
    if (!ok) break;
    host.resize(b.bytes);
    st = copy_sync(ctx, host.data(), b.dev, b.bytes, cudaMemcpyDeviceToHost);
    ok = st == CBL_OK && std::fwrite(host.data(), 1, b.bytes, f) == b.bytes;
  }
  ok = (std::fclose(f) == 0) && ok;
  if (st != CBL_OK) return st;
  if (!ok) return fail(ctx, CBL_ERR_ARG, std::string("write to ") + path + " failed");
  return CBL_OK;
}

cbl_status cbl_load(cbl_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  if (ctx->ready) return fail(ctx, CBL_ERR_STATE, "cbl_load needs a context that is not initialised yet");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, CBL_ERR_ARG, std::string("cannot open ") + path);
  CkptHeader h;
  const CkptHeader mine = ckpt_header(ctx);
  bool ok = std::fread(&h, sizeof(h), 1, f) == 1;
  if (!ok || std::memcmp(h.magic, CKPT_MAGIC, 8) != 0 || h.version != CKPT_VERSION) {
    std::fclose(f);
    return fail(ctx, CBL_ERR_ARG, std::string(path) + " is not a checkpoint of this library version");
  }
  // everything but the step counter must match: parameters, velocity set, precision, bodies, tiles
  CkptHeader a = h, b = mine;
  a.t = b.t = 0;
  a.Lmax = b.Lmax = 0;  // derived from the tiles, compared through the body table below
  if (std::memcmp(&a, &b, sizeof(a)) != 0) {
    std::fclose(f);
    return fail(ctx, CBL_ERR_ARG, "the checkpoint's parameters, velocity set, precision or bodies differ from the context's");
  }
  const int nb = h.nb;
  std::vector<BodyDev> bodies(nb);
  if (nb && std::fread(bodies.data(), sizeof(BodyDev), nb, f) != (size_t)nb) ok = false;
  for (int i = 0; ok && i < nb; ++i)
    for (int k = 0; k < 3; ++k)
      if (bodies[i].L[k] != ctx->hb[i].L[k] || bodies[i].off != ctx->hb[i].off || bodies[i].sz != ctx->hb[i].sz)
        ok = false;
  if (!ok) {
    std::fclose(f);
    return fail(ctx, CBL_ERR_ARG, "the checkpoint's bodies or their tiles differ from the context's");
  }
  const cbl_status sa = alloc_bodies(ctx);
  if (sa != CBL_OK) {
    std::fclose(f);
    return sa;
  }
  ctx->hb = bodies;
  cbl_status st = CBL_OK;
  if (nb) st = copy_sync(ctx, ctx->db, bodies.data(), sizeof(BodyDev) * nb, cudaMemcpyHostToDevice);
  std::vector<char> host;
  for (const Buf& bf : ckpt_buffers(ctx)) {
    if (st != CBL_OK || !ok) break;
    host.resize(bf.bytes);
    ok = std::fread(host.data(), 1, bf.bytes, f) == bf.bytes;
    if (ok) st = copy_sync(ctx, bf.dev, host.data(), bf.bytes, cudaMemcpyHostToDevice);
  }
  std::fclose(f);
  if (st != CBL_OK) return st;
  if (!ok) return fail(ctx, CBL_ERR_ARG, std::string(path) + " is truncated");
  CK(cudaMemsetAsync(ctx->mass_part, 0, (size_t)ctx->n_mass_part * 8, ctx->s));
  if (nb) CK(cudaMemsetAsync(ctx->fsum, 0, sizeof(double) * 6 * nb, ctx->s));  // running sums start anew
  ctx->fsum_steps = 0;
  CK(cudaStreamSynchronize(ctx->s));
  ctx->t = h.t;
  ctx->ready = true;
  ctx->psi_valid = false;
  return CBL_OK;
}

cbl_status cbl_total_mass(cbl_ctx* ctx, double* mass) {
  if (!ctx || !mass) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  if (!ctx->ready) return fail(ctx, CBL_ERR_STATE, "not initialised");
  StepState h;
  CK(cudaMemcpyAsync(&h, ctx->st, sizeof(h), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  *mass = h.last_mass;
  if (!std::isfinite(h.last_mass)) return fail(ctx, CBL_ERR_UNSTABLE, "fluid mass is not finite");
  if (h.err & E_UNSTABLE) return fail(ctx, CBL_ERR_UNSTABLE, "a body update was not finite; the body is held");
  return CBL_OK;
}

cbl_status cbl_info(cbl_ctx* ctx, int* nbodies, int64_t* ncells, int* device_error) {
  if (!ctx) return fail(ctx, CBL_ERR_ARG, "NULL context");
  if (nbodies) *nbodies = (int)ctx->hb.size();
  if (ncells) *ncells = ctx->lat.N;
  if (device_error) {
    StepState h;
    CK(cudaMemcpyAsync(&h, ctx->st, sizeof(h), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    *device_error = h.err;
  }
  return CBL_OK;
}

cbl_status cbl_get_option(cbl_ctx* ctx, const char* key, double* value) {
  if (!ctx || !key || !value) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  const std::string k(key);
  if (k == "lbm_variant") *value = ctx->acc_pass ? 2 : (ctx->fused_tz ? 1 : 0);
  else if (k == "acc_ty") *value = ctx->acc_ty;
  else if (k == "acc_sz") *value = ctx->acc_sz_req > 0 ? ctx->acc_sz_req : ctx->ops.acc_sz(ctx->lat, ctx->prec, ctx->acc_ty, 2);
  else if (k == "fused_ty") *value = ctx->fused_ty;
  else if (k == "fused_tz") *value = ctx->fused_tz;
  else if (k == "lbm_block_x") *value = ctx->block_x;
  else if (k == "node_priority") *value = ctx->node_priority;
  else if (k == "graph_branches") *value = ctx->branches;
  else if (k == "tile_tail") *value = ctx->tile_tail;
  else if (k == "kernel_events") *value = ctx->kev;
  else return fail(ctx, CBL_ERR_ARG, "unknown option " + k);
  return CBL_OK;
}

// z extent of the fused pass's blocks: the requested one, or enough blocks for four waves
static int fused_tz_of(const cbl_ctx* ctx) {
  return ctx->fused_tz_req > 0 ? ctx->fused_tz_req : ctx->ops.fused_tz(ctx->lat, ctx->prec, ctx->fused_ty, 4);
}

cbl_status cbl_set_option(cbl_ctx* ctx, const char* key, double value) {
  if (!ctx || !key) return fail(ctx, CBL_ERR_ARG, "NULL argument");
  const std::string k(key);
  if (k == "lbm_variant") {
    const int v = (int)value;
    if (v != 0 && v != 1 && v != 2) return fail(ctx, CBL_ERR_ARG, "lbm_variant must be 0, 1 or 2");
    ctx->fused_tz = v == 1 ? fused_tz_of(ctx) : 0;
    ctx->acc_pass = v == 2;
  } else if (k == "acc_ty") {
    const int v = (int)value;
    if (v != 8 && v != 16) return fail(ctx, CBL_ERR_ARG, "acc_ty must be 8 or 16");
    ctx->acc_ty = v;
  } else if (k == "acc_sz") {
    const int v = (int)value;
    if (v < 0 || v > ctx->p.nz) return fail(ctx, CBL_ERR_ARG, "acc_sz out of range");
    ctx->acc_sz_req = v;
  } else if (k == "fused_tz") {
    const int v = (int)value;
    if (v < 0 || v > ctx->p.nz) return fail(ctx, CBL_ERR_ARG, "fused_tz out of range");
    ctx->fused_tz_req = v;
    if (ctx->fused_tz) ctx->fused_tz = fused_tz_of(ctx);
  } else if (k == "fused_ty") {
    const int v = (int)value;
    if (v != 4 && v != 8) return fail(ctx, CBL_ERR_ARG, "fused_ty must be 4 or 8");
    ctx->fused_ty = v;
    if (ctx->fused_tz) ctx->fused_tz = fused_tz_of(ctx);
  } else if (k == "node_priority") {
    const int v = (int)value;
    if (v != 0 && v != 1) return fail(ctx, CBL_ERR_ARG, "node_priority must be 0 or 1");
    ctx->node_priority = v;

  } else if (k == "graph_branches") {
    const int v = (int)value;
    if (v != 0 && v != 1) return fail(ctx, CBL_ERR_ARG, "graph_branches must be 0 or 1");
    ctx->branches = v;
  } else if (k == "tile_tail") {
    if (!(value >= 0.0 && value <= 64.0)) return fail(ctx, CBL_ERR_ARG, "tile_tail must be in [0, 64]");
    if (!ctx->hb.empty()) return fail(ctx, CBL_ERR_STATE, "tile_tail must be set before the first body");
    ctx->tile_tail = value;
    return CBL_OK;
  } else if (k == "kernel_events") {
    const int v = (int)value;
    if (v != 0 && v != 1) return fail(ctx, CBL_ERR_ARG, "kernel_events must be 0 or 1");
    if (v && ctx->kev_ring.empty()) {
      for (int k2 = 0; k2 < 2; ++k2) CK(cudaEventCreate(&ctx->kev_cap[k2]));
      ctx->kev_ring.resize(2 * KEV_RING);
      for (cudaEvent_t& e : ctx->kev_ring) CK(cudaEventCreate(&e));
    }
    ctx->kev = v;
    ctx->kev_steps = 0;
  } else if (k == "lbm_block_x") {
    const int v = (int)value;
    if (v != 32 && v != 64 && v != 128) return fail(ctx, CBL_ERR_ARG, "lbm_block_x must be 32, 64 or 128");
    ctx->block_x = v;
  } else {
    return fail(ctx, CBL_ERR_ARG, "unknown option " + k);
  }
  ctx->psi_valid = false;
  if (ctx->gexec) {
    cudaStreamSynchronize(ctx->s);
    cudaGraphExecDestroy(ctx->gexec);
    cudaGraphDestroy(ctx->graph);
    ctx->gexec = nullptr;
    ctx->graph = nullptr;
  }
  return CBL_OK;
}

struct cbl_batch {
  std::vector<cbl_ctx*> ctxs;
  std::vector<cudaStream_t> branches;
  std::vector<cudaEvent_t> events;  // [0] fork, [1..n] joins
  cudaStream_t s = nullptr;
  bool own_stream = false;
  cudaGraph_t graph[2] = {nullptr, nullptr};      // [0] no field record, [1] record fields
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  // persistent mode: one launch of the bulk lattice-Boltzmann pass over every instance, then the
  // instances' side chains on their branches
  int mode = 0;        // 0: one fork/join branch with the whole step per instance; 1: persistent
  int tile_cfg = 1;    // tile shape of the persistent kernel (batch_tile)
  int cooperative = 1;
  int grid = 0;
  long long items = 0;
  long long spin_limit = 4000000000LL;  // clock64 cycles a block may wait at the grid barrier (~2 s)
  BatchInst* tab = nullptr;
  BatchCtl* ctl = nullptr;
};

static cudaError_t batch_capture(cbl_batch* b, int diag, cudaGraph_t* g) {
  cudaError_t e = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  // the instances' kernels run side by side: each sizes its device-sized grids for its share
  LaunchShare share((int)std::min<size_t>(b->ctxs.size(), 64));
  cudaError_t el = cudaSuccess;
  if (b->mode == 1) {
    cbl_ctx* c0 = b->ctxs[0];
    for (cbl_ctx* c : b->ctxs) cudaMemsetAsync(&c->st->diag, diag, sizeof(int), b->s);
    cudaMemsetAsync(b->ctl, 0, BATCH_CTL_RESET_BYTES, b->s);
    el = c0->ops.batch_lbm(c0->prec, b->tile_cfg, b->tab, (int)b->ctxs.size(), b->items, b->ctl, b->grid,
                           b->cooperative, b->s);
  }
  cudaEventRecord(b->events[0], b->s);
  for (size_t k = 0; k < b->ctxs.size(); ++k) {
    cbl_ctx* c = b->ctxs[k];
    cudaStream_t br = b->branches[k];
    cudaStreamWaitEvent(br, b->events[0], 0);
    cudaStream_t keep = c->s;
    const int keep_acc = c->acc_pass;
    c->s = br;
    c->acc_pass = 0;  // a batch runs its instances with the split or fused pass (one psi buffer)
    if (b->mode == 1) {
      enqueue_side_chain(c);
    } else {
      cudaMemsetAsync(&c->st->diag, diag, sizeof(int), br);
      enqueue_step(c);
    }
    c->s = keep;
    c->acc_pass = keep_acc;
    cudaEventRecord(b->events[k + 1], br);
    cudaStreamWaitEvent(b->s, b->events[k + 1], 0);
  }
  cudaError_t e1 = cudaGetLastError();
  cudaError_t e2 = cudaStreamEndCapture(b->s, g);
  if (el != cudaSuccess) return el;
  return e1 != cudaSuccess ? e1 : e2;
}

static void batch_drop_graphs(cbl_batch* b) {
  for (int d = 0; d < 2; ++d) {
    if (b->gexec[d]) cudaGraphExecDestroy(b->gexec[d]);
    if (b->graph[d]) cudaGraphDestroy(b->graph[d]);
    b->gexec[d] = nullptr;
    b->graph[d] = nullptr;
  }
}

// (re)build the instance table and both step graphs for the batch's mode and tile shape
static cudaError_t batch_build(cbl_batch* b) {
  batch_drop_graphs(b);
  if (b->mode == 1) {
    cbl_ctx* c0 = b->ctxs[0];
    int t[3];
    c0->ops.batch_tile(b->tile_cfg, t);
    std::vector<BatchInst> h(b->ctxs.size());
    long long items = 0;
    for (size_t k = 0; k < b->ctxs.size(); ++k) {
      const cbl_ctx* c = b->ctxs[k];
      BatchInst& I = h[k];
      std::memset(&I, 0, sizeof(I));
      I.lat = c->lat;
      I.fa = c->fa;
      I.fb = c->fb;
      I.psi = c->psi;
      I.flags = c->flags;
      I.bodies = c->db;
      I.mass_part = c->mass_part;
      I.st = c->st;
      I.diag_rho = c->diag_rho;
      I.diag_vel = c->diag_vel;
      I.pp = c->pp;
      const int n[3] = {c->lat.nx, c->lat.ny, c->lat.nz};
      for (int a = 0; a < 3; ++a) I.tiles[a] = (n[a] + t[a] - 1) / t[a];
      I.item0 = items;
      items += (long long)I.tiles[0] * I.tiles[1] * I.tiles[2];
    }
    b->items = items;
    cudaError_t e = cudaMemcpy(b->tab, h.data(), sizeof(BatchInst) * h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid = c0->ops.batch_blocks_per_sm(c0->prec, b->tile_cfg) * sms;
    if (b->grid <= 0) return cudaErrorInvalidConfiguration;
    BatchCtl ctl;
    std::memset(&ctl, 0, sizeof(ctl));
    ctl.spin_limit = b->spin_limit;
    e = cudaMemcpy(b->ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  for (int d = 0; d < 2; ++d) {
    cudaError_t e = batch_capture(b, d, &b->graph[d]);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec[d], b->graph[d], cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) {
      cudaGetLastError();
      batch_drop_graphs(b);
      return e;
    }
  }
  return cudaSuccess;
}

cbl_status cbl_batch_create(cbl_ctx* const* ctxs, int n, void* stream, cbl_batch** out) {
  if (!ctxs || n <= 0 || !out) return fail(nullptr, CBL_ERR_ARG, "batch needs contexts");
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k]) return fail(nullptr, CBL_ERR_ARG, "NULL context in batch");
    if (!ctxs[k]->ready) return fail(nullptr, CBL_ERR_STATE, "batch contexts must be initialised");
    // finish whatever the context has queued on its own stream before the batch takes over
    if (cudaStreamSynchronize(ctxs[k]->s) != cudaSuccess) return fail(nullptr, CBL_ERR_CUDA, "sync");
  }
  cbl_batch* b = new cbl_batch();
  b->ctxs.assign(ctxs, ctxs + n);
  // the persistent launch serves instances of one precision and velocity set on the split pass
  bool uniform = true;
  for (int k = 0; k < n; ++k)
    uniform &= ctxs[k]->prec == ctxs[0]->prec && ctxs[k]->ops.q == ctxs[0]->ops.q && ctxs[k]->fused_tz == 0;
  b->mode = uniform ? 1 : 0;
  if (stream) {
    b->s = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return fail(nullptr, CBL_ERR_CUDA, "stream");
    }
    b->own_stream = true;
  }
  b->branches.resize(n);
  b->events.resize(n + 1);
  bool ok = true;
  for (int k = 0; k < n; ++k) ok &= cudaStreamCreateWithFlags(&b->branches[k], cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; k <= n; ++k) ok &= cudaEventCreateWithFlags(&b->events[k], cudaEventDisableTiming) == cudaSuccess;
  ok &= cudaMalloc(&b->tab, sizeof(BatchInst) * n) == cudaSuccess;
  ok &= cudaMalloc(&b->ctl, sizeof(BatchCtl)) == cudaSuccess;
  if (ok && batch_build(b) != cudaSuccess && b->mode == 1) {
    // a cooperative kernel that cannot be captured: the same launch, plain (the grid is sized to be
    // resident, and the barrier's wait is bounded either way)
    b->cooperative = 0;
    ok = batch_build(b) == cudaSuccess;
  } else if (ok) {
    ok = b->gexec[0] != nullptr;
  }
  if (!ok) {
    cudaGetLastError();
    cbl_batch_destroy(b);
    return fail(nullptr, CBL_ERR_CUDA, "batch graph capture failed");
  }
  *out = b;
  return CBL_OK;
}

cbl_status cbl_batch_set_option(cbl_batch* b, const char* key, double value) {
  if (!b || !key) return fail(nullptr, CBL_ERR_ARG, "NULL argument");
  const std::string k(key);
  const int v = (int)value;
  if (cudaStreamSynchronize(b->s) != cudaSuccess) return fail(nullptr, CBL_ERR_CUDA, "sync");
  if (k == "mode") {
    if (v != 0 && v != 1) return fail(nullptr, CBL_ERR_ARG, "mode must be 0 or 1");
    if (v == 1) {
      for (cbl_ctx* c : b->ctxs)
        if (c->prec != b->ctxs[0]->prec || c->ops.q != b->ctxs[0]->ops.q || c->fused_tz)
          return fail(nullptr, CBL_ERR_UNSUPPORTED, "persistent mode needs one precision and velocity set, split pass");
    }
    b->mode = v;
  } else if (k == "tile") {
    if (v < 0 || v >= BATCH_TILE_CFGS) return fail(nullptr, CBL_ERR_ARG, "tile must be 0..3");
    b->tile_cfg = v;
  } else if (k == "spin_limit") {
    if (!(value >= 0)) return fail(nullptr, CBL_ERR_ARG, "spin_limit must be >= 0");
    b->spin_limit = (long long)value;
  } else {
    return fail(nullptr, CBL_ERR_ARG, "unknown batch option " + k);
  }
  if (batch_build(b) != cudaSuccess) return fail(nullptr, CBL_ERR_CUDA, "batch graph capture failed");
  return CBL_OK;
}

cbl_status cbl_batch_info(cbl_batch* b, int* mode, int* tile, long long* items, int* grid) {
  if (!b) return fail(nullptr, CBL_ERR_ARG, "NULL batch");
  if (mode) *mode = b->mode;
  if (tile) *tile = b->tile_cfg;
  if (items) *items = b->items;
  if (grid) *grid = b->grid;
  return CBL_OK;
}

cbl_status cbl_batch_step(cbl_batch* b, int nsteps) {
  if (!b) return fail(nullptr, CBL_ERR_ARG, "NULL batch");
  if (nsteps < 0) return fail(nullptr, CBL_ERR_ARG, "nsteps must be >= 0");
  for (int k = 0; k < nsteps; ++k)
    if (cudaGraphLaunch(b->gexec[k == nsteps - 1 ? 1 : 0], b->s) != cudaSuccess)
      return fail(nullptr, CBL_ERR_CUDA, "batch graph launch failed");
  for (cbl_ctx* c : b->ctxs) {
    c->t += nsteps;
    c->fsum_steps += nsteps;
    c->psi_valid = false;
  }
  return CBL_OK;
}

cbl_status cbl_batch_sync(cbl_batch* b) {
  if (!b) return fail(nullptr, CBL_ERR_ARG, "NULL batch");
  if (cudaStreamSynchronize(b->s) != cudaSuccess) return fail(nullptr, CBL_ERR_CUDA, "sync");
  if (b->mode == 1) {
    int err = 0;
    if (cudaMemcpy(&err, &b->ctl->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(nullptr, CBL_ERR_CUDA, "sync");
    if (err) {
      const int zero = 0;
      cudaMemcpy(&b->ctl->err, &zero, sizeof(int), cudaMemcpyHostToDevice);
      return fail(nullptr, CBL_ERR_TIMEOUT, "a grid-barrier wait of the persistent batch kernel ran out");
    }
  }
  return CBL_OK;
}

cbl_status cbl_batch_destroy(cbl_batch* b) {
  if (!b) return CBL_OK;
  if (b->s) cudaStreamSynchronize(b->s);
  batch_drop_graphs(b);
  for (cudaStream_t br : b->branches)
    if (br) cudaStreamDestroy(br);
  for (cudaEvent_t e : b->events)
    if (e) cudaEventDestroy(e);
  if (b->tab) cudaFree(b->tab);
  if (b->ctl) cudaFree(b->ctl);
  if (b->own_stream) cudaStreamDestroy(b->s);
  delete b;
  return CBL_OK;
}

cbl_status cbl_destroy(cbl_ctx* ctx) {
  if (!ctx) return CBL_OK;
  cudaStreamSynchronize(ctx->s);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  dfree_all(ctx);
  if (ctx->own_stream) cudaStreamDestroy(ctx->s);
  cudaStreamDestroy(ctx->side);
  cudaEventDestroy(ctx->ev_fork);
  cudaEventDestroy(ctx->ev_join);
  for (cudaEvent_t e : ctx->kev_cap)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->kev_ring)
    if (e) cudaEventDestroy(e);
  delete ctx;
  return CBL_OK;
}

}  // extern "C"
