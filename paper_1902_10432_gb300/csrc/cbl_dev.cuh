// Internal device-side definitions of the capillary-bridge library (not part of the C ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "periodic.h"
#include "weights.h"

namespace cbl {

// ------------------------------------------------------------------------------------------
// Velocity sets. D3Q27 is the set the paper prints (Sec. 3.2.1): weights 8/27 (rest), 2/27 (faces),
// 1/54 (edges), 1/216 (corners). D3Q19 is its textbook |c|^2 <= 2 subset with weights 1/3, 1/18,
// 1/36. Order: rest, +-x, +-y, +-z, the 12 edge directions, then (D3Q27) the 8 corners; each odd
// index i is followed by its opposite, so opp(i) = i + 1 for odd i and i - 1 for even i > 0 in both
// sets. The lattice-Boltzmann kernels are compiled once per set, in namespace q19 or q27.
namespace q19 {
constexpr int Q = 19;
__host__ __device__ constexpr int cx_of(int i) {
  constexpr int v[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
  return v[i];
}
__host__ __device__ constexpr int cy_of(int i) {
  constexpr int v[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
  return v[i];
}
__host__ __device__ constexpr int cz_of(int i) {
  constexpr int v[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
  return v[i];
}
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr double w_of(int i) {
  return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}
}  // namespace q19

namespace q27 {
constexpr int Q = 27;
__host__ __device__ constexpr int cx_of(int i) {
  constexpr int v[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
  return v[i];
}
__host__ __device__ constexpr int cy_of(int i) {
  constexpr int v[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, -1, 1, 1, -1};
  return v[i];
}
__host__ __device__ constexpr int cz_of(int i) {
  constexpr int v[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, 1, -1};
  return v[i];
}
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr double w_of(int i) {
  return i == 0 ? 8.0 / 27.0 : (i <= 6 ? 2.0 / 27.0 : (i <= 18 ? 1.0 / 54.0 : 1.0 / 216.0));
}
}  // namespace q27

// Cell flags (uint16): bit 15 solid, bit 14 "became solid in the last flag update" (cover
// event, consumed by the refill), bit 13 "fluid cell with a solid neighbour along a lattice
// direction" (set by the refill pass), bits 0..12 owner body id of a solid cell.
constexpr uint16_t F_SOLID = 0x8000;
constexpr uint16_t F_COVER = 0x4000;
constexpr uint16_t F_NEAR = 0x2000;
constexpr uint16_t F_OWNER = 0x1FFF;
constexpr int MAX_BODIES = 0x1FFF;
constexpr uint16_t F_STALE = 0x1FFF;  // owner id of a cell solid before a body move (never a body)
constexpr int MAXNB = 24;  // neighbour-list capacity per body (tiles that overlap)
// Per-body member record (rebuilt by the refill pass from the cells with phi >= the membership
// threshold): tile-coordinate box lo[3], hi[3], then the bit pattern of the largest squared distance
// of a member cell from the body's centre X (a non-negative float: its bits order like the value),
// and one unused word.
constexpr int MBOX_N = 8, MBOX_R2 = 6;

// Fluid-mass accumulation slots written by the collision kernel and summed by the body kernel.
constexpr int MASS_SLOTS = 256;

// Device error word bits.
// E_UNSTABLE: a body's update gave a non-finite position, velocity or angular velocity, or moved it
// by a lattice length or more in one step; that body is then held at its last pose.
constexpr int E_TILE = 1, E_NBLIST = 2, E_REFILL = 4, E_UNSTABLE = 8;

struct Lat {
  int nx, ny, nz;
  long long N;   // cells
  long long Ns;  // distance between the population arrays of two directions, >= N (padded)
};

// Padding of the population stride: with N a large power of two the 19 direction arrays would all
// start at the same DRAM channel offset; an odd multiple of 128 elements spreads them.
#ifndef CBL_POP_PAD
#define CBL_POP_PAD 1152
#endif
inline long long pop_stride(long long N) { return ((N + 127) / 128) * 128 + CBL_POP_PAD; }

// One solid body: rigid state (FP64), shape for the initial profile, and its phase-field tile.
// The tile is a box of L cells per axis whose cell (i,j,k) holds the global cell
// ((o + (i,j,k)) mod n); cells outside the tile have phi = 0. Three buffers of `sz` doubles start
// at `off` in the arena: buffer 0 is the current field.
struct BodyDev {
  double X[3], Xprev[3], V[3], W[3], Q[4];
  double M, Ib[9], Ibinv[9];  // body-frame inertia and its inverse
  double wet, psi_wet, vol_ref, rho_s;
  float psi_wet_f;  // psi_wet rounded once on the host for the FP32 kernels
  // X, V, W rounded to float for the FP32 kernels' wall terms (mirror_f after every update)
  float Xf[3], Vf[3], Wf[3];
  double c0[3], radius, half[3], q0[4];
  int fixed, shape;
  int rot_lock;  // bit c: angular velocity component c held at zero (body spans the lattice)
  int o[3], o_prev[3], L[3];
  long long off, sz;
  int nnb;
  int nbl[MAXNB];
};

__host__ __device__ inline void mirror_f(BodyDev& b) {
  for (int a = 0; a < 3; ++a) {
    b.Xf[a] = (float)b.X[a];
    b.Vf[a] = (float)b.V[a];
    b.Wf[a] = (float)b.W[a];
  }
}

// Per-step accumulator layout per body (18 doubles).
constexpr int ACC_MOM_F = 0, ACC_MOM_T = 3, ACC_ADH_F = 6, ACC_ADH_T = 9, ACC_REP_F = 12,
              ACC_REP_T = 15, ACC_N = 18;

struct StepState {
  int parity;   // which population buffer is the source this step
  int diag;     // 1: the collision writes rho and v
  int err;      // error word
  int psi_skip;  // accumulating pass: psi of this step came from a whole-lattice density pass
  double mass;       // fluid mass of the current step (accumulating)
  double last_mass;  // fluid mass of the last completed step
  unsigned long long lost_refills;
  unsigned nbnd;     // entries of the boundary-cell list (fluid cells next to a solid)
  unsigned ncover;   // nodes covered in this step's flag update
};

struct PhysParams {
  double tau, G, rho0;
  double ext[3];
  double eta, mobility, sigma_sf, sigma_ss;
  double e0, rc;
  int nrep;
  double solid_threshold, member_threshold;
  int mpf;
  // FP32 copies for the FP32 kernels, rounded once on the host (fill_float_params): a per-thread
  // double-to-float conversion is an FP64-pipe instruction, and GB300 issues FP64 at 1/64 rate
  float tau_f, G_f, rho0_f, ext_f[3];
};

inline void fill_float_params(PhysParams& p) {
  p.tau_f = (float)p.tau;
  p.G_f = (float)p.G;
  p.rho0_f = (float)p.rho0;
  for (int k = 0; k < 3; ++k) p.ext_f[k] = (float)p.ext[k];
}

// a parameter in the working precision R: the double itself, or its host-rounded float copy
template <typename R>
__device__ __forceinline__ R par(double d, float f);
template <>
__device__ __forceinline__ double par<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float par<float>(double, float f) { return f; }

// Bit-pattern tests of doubles on the integer pipe (GB300 issues FP64 at a small fraction of the
// FP32 rate). For any double v and a positive threshold t: v > t <=> bits(v) > bits(t) as signed
// 64-bit integers, since negative v have the sign bit set.
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }

// wrapi, mimg, wrapd: periodic wraps with a fixed operation count (periodic.h)

// ---- batches of independent lattices -----------------------------------------------------------
// One instance of a batch, as the persistent lattice-Boltzmann kernel sees it (a device-resident
// table, one entry per instance): its lattice and buffers, and where its work items start. A work
// item is one tile of TX x TY x TZ cells of one instance; the items of all instances are numbered
// one after the other, instance by instance.
struct BatchInst {
  Lat lat;
  void *fa, *fb, *psi;
  const uint16_t* flags;
  const BodyDev* bodies;
  double* mass_part;
  StepState* st;
  double *diag_rho, *diag_vel;
  PhysParams pp;
  int tiles[3];    // tiles per axis
  int pad;
  long long item0;  // first work item of this instance
};

// Control block of the persistent kernel. queue[p]: next work item of phase p; arrive / gen: the
// grid barrier between the phases (arrivals of this generation, generation count); spin_limit: the
// longest a block waits at the barrier, in clock64 cycles, before it sets err bit 0 and returns.
// The first 20 bytes (queues and arrivals) are cleared before every launch.
struct BatchCtl {
  unsigned long long queue[2];
  unsigned arrive, gen;
  long long spin_limit;
  int err, pad;
};
constexpr size_t BATCH_CTL_RESET_BYTES = 2 * sizeof(unsigned long long) + sizeof(unsigned);
constexpr int BATCH_TILE_CFGS = 4;  // tile shapes of the persistent kernel (see batch_tile)

// Share of the GPU that the kernels launched by this host thread may assume (1 = all of it). The
// grid-stride kernels whose work is only known on the device (the collision of the cells next to a
// solid, the solid-fluid force pass, the repulsion) size their grids for a few waves of the whole
// GPU; a batch that runs n instances side by side sets n while it captures their steps, so that the
// n copies together fill the GPU instead of each filling it (capi.cu: LaunchShare).
extern thread_local int g_launch_share;

// ---- kernel launchers (defined in lbm.cu / lbm27.cu per velocity set, and phase.cu) ------------
// Populations live in two buffers fa, fb; StepState::parity selects the current state
// (0: fa, 1: fb). The step reads the current buffer, writes the other, and the closing kernel flips
// the parity, so one captured graph serves every step.
// launch_lbm_step phases: bit 0 density, bit 1 bulk collision, bit 2 collision of the cells next to
// a solid. launch_lbm_fused: density and bulk collision in one pass (cells next to a solid excluded:
// launch_density_tiles fills psi over the bodies' tiles for their collision); blocks of 32 x ty
// consumer columns (ty 4 or 8) and as many producer threads, marching tz planes along z.
#define CBL_LBM_LAUNCHERS                                                                              \
  void set_fp16_weights(cudaStream_t s);                                                             \
  void launch_lbm_step(int prec, const Lat& lat, void* fa, void* fb, const uint16_t* flags, void* psi, \
                       void* psi_b, const BodyDev* bodies, double* mass_part, unsigned blocks,        \
                       StepState* st, double* diag_rho, double* diag_vel, const PhysParams& pp,       \
                       void* nbuf, const int* blist, cudaStream_t s, int phases);                     \
  int acc_sz(const Lat& lat, int prec, int ty, int waves);                                          \
  cudaError_t launch_lbm_acc(int prec, const Lat& lat, void* fa, void* fb, const uint16_t* flags,    \
                             void* psi_a, void* psi_b, void* rhop, const BodyDev* bodies,           \
                             double* mass_part, StepState* st, double* diag_rho, double* diag_vel,  \
                             const PhysParams& pp, int ty, int sz, cudaStream_t s);                 \
  void launch_psi_fixup(int prec, const Lat& lat, const void* fa, const void* fb, void* psi_a,       \
                        void* psi_b, const void* rhop, const StepState* st, const PhysParams& pp,    \
                        int ty, int sz, cudaStream_t s);                                             \
  int fused_tz(const Lat& lat, int prec, int ty, int waves);                                        \
  void launch_lbm_fused(int prec, const Lat& lat, void* fa, void* fb, const uint16_t* flags,         \
                        const BodyDev* bodies, double* mass_part, StepState* st, double* diag_rho,   \
                        double* diag_vel, const PhysParams& pp, int tz, int ty, cudaStream_t s);     \
  void launch_density_tiles(int prec, const Lat& lat, const void* fa, const void* fb,                \
                            const StepState* st, const uint16_t* flags, const BodyDev* bodies, int nb, \
                            int max_tile, void* psi, void* psi_b, const PhysParams& pp,              \
                            cudaStream_t s);                                                         \
  void launch_boundary(int prec, const Lat& lat, const void* fa, const void* fb, const uint16_t* flags, \
                       const BodyDev* bodies, int nb, double* acc, const int* blist, const StepState* st, \
                       const void* nbuf, double G, cudaStream_t s);                                   \
  void launch_read_populations(int prec, const Lat& lat, const void* fa, const void* fb,             \
                               const StepState* st, const uint16_t* flags, double* out, cudaStream_t s); \
  void launch_zero_solid(int prec, const Lat& lat, void* fa, void* fb, const StepState* st,          \
                         const uint16_t* flags, const BodyDev* bodies, int nb, int max_tile,         \
                         cudaStream_t s);                                                             \
  void launch_init_fluid(int prec, const Lat& lat, void* fa, const uint16_t* flags, const double* rho, \
                         const double* u, cudaStream_t s);                                            \
  void launch_refill(int prec, const Lat& lat, void* fa, void* fb, uint16_t* flags, const BodyDev* bodies, \
                     int nb, int max_tile, StepState* st, int* blist, const double* arena,           \
                     double member_thr, int* mbox, int next, cudaStream_t s);                        \
  void batch_tile(int cfg, int* t);                                                                   \
  int batch_blocks_per_sm(int prec, int cfg);                                                         \
  cudaError_t launch_batch_lbm(int prec, int cfg, const BatchInst* tab, int ninst, long long items,  \
                               BatchCtl* ctl, int grid, int cooperative, cudaStream_t s);
namespace q19 {
CBL_LBM_LAUNCHERS
}
namespace q27 {
CBL_LBM_LAUNCHERS
}

// The launchers of one velocity set, chosen when a context is created.
struct LbmOps {
  int q;
  decltype(&q19::set_fp16_weights) set_fp16_weights;
  decltype(&q19::launch_lbm_step) lbm_step;
  decltype(&q19::acc_sz) acc_sz;
  decltype(&q19::launch_lbm_acc) lbm_acc;
  decltype(&q19::launch_psi_fixup) psi_fixup;
  decltype(&q19::fused_tz) fused_tz;
  decltype(&q19::launch_lbm_fused) lbm_fused;
  decltype(&q19::launch_density_tiles) density_tiles;
  decltype(&q19::launch_boundary) boundary;
  decltype(&q19::launch_read_populations) read_populations;
  decltype(&q19::launch_zero_solid) zero_solid;
  decltype(&q19::launch_init_fluid) init_fluid;
  decltype(&q19::launch_refill) refill;
  decltype(&q19::batch_tile) batch_tile;
  decltype(&q19::batch_blocks_per_sm) batch_blocks_per_sm;
  decltype(&q19::launch_batch_lbm) batch_lbm;
};
inline LbmOps lbm_ops(int q) {
#define CBL_OPS(ns) \
  LbmOps { q, &ns::set_fp16_weights, &ns::launch_lbm_step, &ns::acc_sz, &ns::launch_lbm_acc,                     \
           &ns::launch_psi_fixup, &ns::fused_tz, &ns::launch_lbm_fused,                                             \
           &ns::launch_density_tiles, &ns::launch_boundary,                                                             \
           &ns::launch_read_populations, &ns::launch_zero_solid, &ns::launch_init_fluid, &ns::launch_refill,        \
           &ns::batch_tile, &ns::batch_blocks_per_sm, &ns::launch_batch_lbm }
  return q == 27 ? CBL_OPS(q27) : CBL_OPS(q19);
#undef CBL_OPS
}

void launch_clear_tile_flags(const Lat& lat, const BodyDev* bodies, int nb, int max_tile, uint16_t* flags,
                             cudaStream_t s);
void launch_clear_stale(const Lat& lat, uint16_t* flags, cudaStream_t s);
void launch_reset_member_boxes(int* mbox, int nb, cudaStream_t s);
void launch_rasterize(const Lat& lat, BodyDev* bodies, int nb, int max_tile, double* arena,
                      double eta, cudaStream_t s);
void launch_neighbour_lists(BodyDev* bodies, int nb, const Lat& lat, StepState* st, cudaStream_t s);
void launch_flags(const Lat& lat, BodyDev* bodies, int nb, int max_tile, double* arena, uint16_t* flags,
                  double threshold, int init, StepState* st, cudaStream_t s);
void launch_body_props(const Lat& lat, BodyDev* bodies, int nb, int max_tile, double* arena,
                       double* scratch, cudaStream_t s);
void launch_repulsion(const Lat& lat, const BodyDev* bodies, int nb, int max_tile, const double* arena, double* acc,
                      const PhysParams& pp, const int* mbox, cudaStream_t s);
void launch_bodies(const Lat& lat, BodyDev* bodies, int nb, double* acc, double* last, double* volacc,
                   StepState* st, double* rtab, int Lmax, int* mbox, double* fsum, cudaStream_t s);
void launch_finish(double* mass_part, unsigned n_mass_part, StepState* st, cudaStream_t s);
void launch_advect(const Lat& lat, const BodyDev* bodies, int nb, int max_tile, double* arena, int mpf, double* volacc,
                   StepState* st, const double* rtab, int Lmax, cudaStream_t s);
void set_repulsion_offsets(double rc, double e0, int nrep, cudaStream_t s);
void launch_kinetics(const Lat& lat, const BodyDev* bodies, int nb, int max_tile, double* arena,
                     const double* volacc, const PhysParams& pp, cudaStream_t s);
void launch_phi_dense(const Lat& lat, const BodyDev* bodies, int nb, int max_tile, const double* arena,
                      int body, double* out, cudaStream_t s);

}  // namespace cbl
