// Solid-body kernels of the capillary-bridge step (Sec. 3.1 and 3.3 of arXiv:1902.10432).
//
// Each body's phase field lives in a tile (a box of the periodic lattice that follows the body);
// phi is zero outside it. All phase-field arithmetic, reductions and the rigid-body update are FP64.
//  k_rasterize    : initial profile 1/2 - 1/2 sin(pi d / eta) of the signed distance d (Sec. 3.1).
//  k_flags        : clamp to [0,1], renormalise the solid sum, obstacle flag (fluid phase below the
//                   threshold, Sec. 3.2.2), owner = argmax, cover events.
//  k_body_props   : mass, centre of mass and inertia from phi.
//  k_repulsion    : solid-solid repulsion between body points (Eqs. soild_solid_potential and
//                   solid_solid_force, Sec. 3.1.2).
//  k_bodies       : force/torque totals and the rigid-body update (Sec. 3.1.1), tile recentring,
//                   overlap lists, fluid-mass total.
//  k_sweep        : one conservative MUSCL sweep with the monotonized-central limiter of
//                   d(phi)/dt = -u_B . grad(phi) (Eq. phase_advection, Sec. 3.3), x, y, z in turn.
//  k_kinetics     : Eq. sim_proc_phase_field_dynamics with the volume-restoring Delta g (Sec. 3.3).
#include <climits>
#include "cbl_dev.cuh"

namespace cbl {

constexpr double PI = 3.14159265358979323846;
// A phase counts as present where phi > PHI_EPS; the clamp sets phi < PHI_EPS to 0 and
// phi > 1 - PHI_EPS to 1. This keeps "present" (which sets N in the kinetics) from hinging on the
// last bit of a rounding, and keeps the support of a moving field compact.
constexpr double PHI_EPS = 1e-12;
constexpr int MAXOFF = 512;
__constant__ int c_off[3 * MAXOFF];
__constant__ double c_offf[3 * MAXOFF];  // force on the first point of a pair at offset d: f(d)
__constant__ int c_noff;

// Offsets d with 0 < |d| < r_c and the pair force e0 (n / r_c) |(|d| - r_c) / r_c|^(n-1) (-d/|d|)
// (Eq. solid_solid_force) that a point feels from a point at x + d.
void set_repulsion_offsets(double rc, double e0, int nrep, cudaStream_t s) {
  int off[3 * MAXOFF];
  double ff[3 * MAXOFF];
  int n = 0;
  int R = (int)ceil(rc);
  for (int dz = -R; dz <= R; ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        int d2 = dx * dx + dy * dy + dz * dz;
        if (d2 > 0 && (double)d2 < rc * rc && n < MAXOFF) {
          off[3 * n] = dx;
          off[3 * n + 1] = dy;
          off[3 * n + 2] = dz;
          const double d = sqrt((double)d2);
          const double mag = e0 * nrep / rc * pow(fabs((d - rc) / rc), (double)(nrep - 1));
          ff[3 * n] = -dx / d * mag;
          ff[3 * n + 1] = -dy / d * mag;
          ff[3 * n + 2] = -dz / d * mag;
          n++;
        }
      }
  cudaMemcpyToSymbolAsync(c_off, off, sizeof(int) * 3 * n, 0, cudaMemcpyHostToDevice, s);
  cudaMemcpyToSymbolAsync(c_offf, ff, sizeof(double) * 3 * n, 0, cudaMemcpyHostToDevice, s);
  cudaMemcpyToSymbolAsync(c_noff, &n, sizeof(int), 0, cudaMemcpyHostToDevice, s);
}

// ---- tile helpers ------------------------------------------------------------------------------
struct TileCell {
  int i0, i1, i2;  // tile-local
  int gx, gy, gz;  // global (wrapped)
};

__device__ __forceinline__ TileCell tile_cell(const BodyDev& b, long long t, const Lat& lat) {
  TileCell c;
  const unsigned u = (unsigned)t, L0 = (unsigned)b.L[0], L1 = (unsigned)b.L[1];  // tiles hold < 2^31 cells
  const unsigned r = u / L0;
  c.i0 = (int)(u - r * L0);
  c.i1 = (int)(r % L1);
  c.i2 = (int)(r / L1);
  c.gx = wrapi_near(b.o[0] + c.i0, lat.nx);
  c.gy = wrapi_near(b.o[1] + c.i1, lat.ny);
  c.gz = wrapi_near(b.o[2] + c.i2, lat.nz);
  return c;
}

// local index of global cell g in a tile with origin o, or -1 if outside
__device__ __forceinline__ long long tile_index(const int o[3], const int L[3], int gx, int gy, int gz, const Lat& lat) {
  int a = wrapi_near(gx - o[0], lat.nx), b = wrapi_near(gy - o[1], lat.ny), c = wrapi_near(gz - o[2], lat.nz);
  if (a >= L[0] || b >= L[1] || c >= L[2]) return -1;
  return (long long)a + (long long)L[0] * ((long long)b + (long long)L[1] * c);
}

__device__ __forceinline__ double phi_at(const double* buf, const BodyDev& b, int gx, int gy, int gz, const Lat& lat) {
  long long k = tile_index(b.o, b.L, gx, gy, gz, lat);
  return k < 0 ? 0.0 : buf[k];
}

__device__ __forceinline__ bool covered_by_lower_body(const BodyDev* bodies, const BodyDev& b, int self, int gx, int gy,
                                                      int gz, const Lat& lat) {
  for (int k = 0; k < b.nnb; ++k) {
    int o = b.nbl[k];
    if (o >= self) break;
    if (tile_index(bodies[o].o, bodies[o].L, gx, gy, gz, lat) >= 0) return true;
  }
  return false;
}

__device__ __forceinline__ void quat_R(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

__device__ __forceinline__ void xcross(const double a[3], const double b[3], double r[3]) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ double dwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- initial profile ---------------------------------------------------------------------------
__device__ double body_sdf(const BodyDev& b, const double r[3]) {
  if (b.shape == 0) return sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) - b.radius;
  double R[9];
  quat_R(b.q0, R);
  double o = 0, m = -1e300;
  for (int a = 0; a < 3; ++a) {
    double l = R[0 + a] * r[0] + R[3 + a] * r[1] + R[6 + a] * r[2];
    double q = fabs(l) - b.half[a];
    double v = q > 0 ? q : 0;
    o += v * v;
    m = q > m ? q : m;
  }
  return sqrt(o) + (m < 0 ? m : 0.0);
}

__global__ void k_rasterize(BodyDev* bodies, double* arena, Lat lat, double eta) {
  const BodyDev& b = bodies[blockIdx.y];
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b.sz) return;
  TileCell c = tile_cell(b, t, lat);
  double r[3] = {mimg(c.gx - b.c0[0], lat.nx), mimg(c.gy - b.c0[1], lat.ny), mimg(c.gz - b.c0[2], lat.nz)};
  double d = body_sdf(b, r);
  double v = d <= -0.5 * eta ? 1.0 : (d >= 0.5 * eta ? 0.0 : 0.5 - 0.5 * sin(PI * d / eta));
  double* buf = arena + b.off;
  buf[t] = v;
  buf[b.sz + t] = 0.0;
  buf[2 * b.sz + t] = 0.0;
}

// ---- overlap lists -----------------------------------------------------------------------------
__device__ bool tiles_overlap(const BodyDev& a, const BodyDev& b, const Lat& lat) {
  const int n[3] = {lat.nx, lat.ny, lat.nz};
  for (int d = 0; d < 3; ++d) {
    bool ov = wrapi_near(b.o[d] - a.o[d], n[d]) < a.L[d] || wrapi_near(a.o[d] - b.o[d], n[d]) < b.L[d];
    if (!ov) return false;
  }
  return true;
}

__device__ void build_lists(BodyDev* bodies, int nb, const Lat& lat, StepState* st) {
  for (int a = threadIdx.x; a < nb; a += blockDim.x) {
    int cnt = 0;
    for (int b = 0; b < nb; ++b) {
      if (b == a || !tiles_overlap(bodies[a], bodies[b], lat)) continue;
      if (cnt < MAXNB) bodies[a].nbl[cnt++] = b;
      else atomicOr(&st->err, E_NBLIST);
    }
    bodies[a].nnb = cnt;
  }
}

__global__ void k_neighbour_lists(BodyDev* bodies, int nb, Lat lat, StepState* st) {
  build_lists(bodies, nb, lat, st);
}

// ---- flags --------------------------------------------------------------------------------------
__global__ void k_flags(BodyDev* bodies, double* arena, uint16_t* flags, Lat lat, double thr, int init,
                        StepState* st) {
  const int self = blockIdx.y;
  const BodyDev& b = bodies[self];
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b.sz) return;
  TileCell c = tile_cell(b, t, lat);
  if (b.nnb && covered_by_lower_body(bodies, b, self, c.gx, c.gy, c.gz, lat)) return;
  const long long n_cell = c.gx + (long long)lat.nx * (c.gy + (long long)lat.ny * c.gz);
  bool shared = false;
  for (int k = 0; k < b.nnb && !shared; ++k) {
    const BodyDev& o = bodies[b.nbl[k]];
    shared = tile_index(o.o, o.L, c.gx, c.gy, c.gz, lat) >= 0;
  }
  if (!shared) {
    // this body alone: the general form below with one phase (S = phi after the clamp, which
    // cannot exceed 1), without its per-phase arrays
    double* p0 = arena + b.off + t;
    const long long vb = dbits(*p0);
    double S;
    if (vb == 0 || vb == dbits(1.0)) {
      S = vb == 0 ? 0.0 : 1.0;  // unchanged by the clamp and the flush
    } else {
      double v = fmin(1.0, fmax(0.0, *p0));
      if (v < PHI_EPS) v = 0.0;
      if (v > 1.0 - PHI_EPS) v = 1.0;
      *p0 = v;
      S = v;
    }
    uint16_t nf = 0;
    if (1.0 - S < thr) {
      nf = F_SOLID | (uint16_t)self;
      if (!init && !(flags[n_cell] & F_SOLID)) {
        nf |= F_COVER;
        atomicAdd(&st->ncover, 1u);
      }
    }
    flags[n_cell] = nf;
    return;
  }
  // bodies covering this cell, ascending id (self is the lowest)
  double* ptr[MAXNB + 1];
  int ids[MAXNB + 1];
  int m = 0;
  ptr[m] = arena + b.off + t;
  ids[m++] = self;
  for (int k = 0; k < b.nnb; ++k) {
    const BodyDev& o = bodies[b.nbl[k]];
    long long j = tile_index(o.o, o.L, c.gx, c.gy, c.gz, lat);
    if (j >= 0) {
      ptr[m] = arena + o.off + j;
      ids[m++] = b.nbl[k];
    }
  }
  double S = 0.0;
  for (int k = 0; k < m; ++k) {
    double v = *ptr[k];
    v = fmin(1.0, fmax(0.0, v));
    if (v < PHI_EPS) v = 0.0;
    if (v > 1.0 - PHI_EPS) v = 1.0;
    *ptr[k] = v;
    S += v;
  }
  if (S > 1.0) {
    double S2 = 0.0;
    for (int k = 0; k < m; ++k) {
      double v = *ptr[k] / S;
      *ptr[k] = v;
      S2 += v;
    }
    S = S2;
  }
  const long long n = c.gx + (long long)lat.nx * (c.gy + (long long)lat.ny * c.gz);
  uint16_t old = flags[n];
  uint16_t nf = 0;
  if (1.0 - S < thr) {
    int best = ids[0];
    double bv = *ptr[0];
    for (int k = 1; k < m; ++k)
      if (*ptr[k] > bv) {
        bv = *ptr[k];
        best = ids[k];
      }
    nf = F_SOLID | (uint16_t)best;
    if (!init && !(old & F_SOLID)) {
      nf |= F_COVER;
      atomicAdd(&st->ncover, 1u);
    }
  }
  flags[n] = nf;
}

// ---- body properties (initialisation) ---------------------------------------------------------
// pass 0: sum phi and sum r phi about the nominal centre; pass 1: inertia about X
__global__ void k_body_props(const BodyDev* bodies, const double* arena, double* scratch, Lat lat, int pass) {
  const int self = blockIdx.y;
  const BodyDev& b = bodies[self];
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  TileCell c;
  if (t < b.sz) {
    c = tile_cell(b, t, lat);
    v = arena[b.off + t];
  }
  double a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (v != 0.0) {
    if (pass == 0) {
      a[0] = v;
      a[1] = v * mimg(c.gx - b.c0[0], lat.nx);
      a[2] = v * mimg(c.gy - b.c0[1], lat.ny);
      a[3] = v * mimg(c.gz - b.c0[2], lat.nz);
    } else {
      double r[3] = {mimg(c.gx - b.X[0], lat.nx), mimg(c.gy - b.X[1], lat.ny), mimg(c.gz - b.X[2], lat.nz)};
      double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) a[3 * p + q] = v * ((p == q ? rr : 0.0) - r[p] * r[q]);
    }
  }
  for (int k = 0; k < 9; ++k) {
    double s = dwarp_sum(a[k]);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(scratch + self * 9 + k, s);
  }
}

__global__ void k_body_props_finish(BodyDev* bodies, int nb, const double* scratch, Lat lat, int pass) {
  int self = blockIdx.x * blockDim.x + threadIdx.x;
  if (self >= nb) return;
  BodyDev& b = bodies[self];
  const double* s = scratch + self * 9;
  const int n[3] = {lat.nx, lat.ny, lat.nz};
  if (pass == 0) {
    for (int a = 0; a < 3; ++a) {
      double X = b.c0[a] + s[1 + a] / s[0];
      X = fmod(X, (double)n[a]);
      if (X < 0) X += n[a];
      b.X[a] = X;
      b.Xprev[a] = X;
    }
    mirror_f(b);
    b.M = b.rho_s * s[0];
    b.vol_ref = s[0];
  } else {
    double R[9];
    quat_R(b.Q, R);
    const double rho_s = b.rho_s;
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) {
        double acc = 0;
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) acc += R[3 * k + a] * (rho_s * s[3 * k + l]) * R[3 * l + c];
        b.Ib[3 * a + c] = acc;
      }
    const double* I = b.Ib;
    const double det = I[0] * (I[4] * I[8] - I[5] * I[7]) - I[1] * (I[3] * I[8] - I[5] * I[6]) +
                       I[2] * (I[3] * I[7] - I[4] * I[6]);
    b.Ibinv[0] = (I[4] * I[8] - I[5] * I[7]) / det;
    b.Ibinv[1] = (I[2] * I[7] - I[1] * I[8]) / det;
    b.Ibinv[2] = (I[1] * I[5] - I[2] * I[4]) / det;
    b.Ibinv[3] = (I[5] * I[6] - I[3] * I[8]) / det;
    b.Ibinv[4] = (I[0] * I[8] - I[2] * I[6]) / det;
    b.Ibinv[5] = (I[2] * I[3] - I[0] * I[5]) / det;
    b.Ibinv[6] = (I[3] * I[7] - I[4] * I[6]) / det;
    b.Ibinv[7] = (I[1] * I[6] - I[0] * I[7]) / det;
    b.Ibinv[8] = (I[0] * I[4] - I[1] * I[3]) / det;
  }
}

// ---- solid-solid repulsion ---------------------------------------------------------------------
// For a point x of body A (phi_A >= the membership threshold) and every body B whose tile overlaps
// A's: sum the table forces f(d) over the points x + d of B; torque (x - X_A) x (sum f).

__global__ void __launch_bounds__(256) k_repulsion(const BodyDev* bodies, const double* arena, double* acc, Lat lat,
                                                   double rc, int Rc, double thr, double eta,
                                                   const int* __restrict__ mbox) {
  const int self = blockIdx.y;
  const BodyDev& a = bodies[self];
  if (a.nnb == 0) return;  // block-uniform
  // block-uniform cull: member points (phi >= 1/2) lie within the support of the profile, the
  // shape's bounding sphere grown by eta/2; no pair can be within rc unless two such spheres are
  // and the member boxes: every member point of A lies in A's box, so if along some axis the two
  // boxes are more than Rc cells apart (periodic distance), no point of A passes the per-point box
  // test below
  __shared__ int s_near;
  if (threadIdx.x == 0) {
    int nearby = 0;
    const int nn[3] = {lat.nx, lat.ny, lat.nz};
    const int* ba = mbox + MBOX_N * self;
    // every member point of a body lies within its member radius of its centre X, so two bodies
    // whose centres are farther apart than the two member radii plus rc (and a cell of slack) have
    // no pair in range
    const double ra = sqrt((double)__int_as_float(ba[MBOX_R2]));
    for (int k = 0; k < a.nnb && !nearby; ++k) {
      const BodyDev& b = bodies[a.nbl[k]];
      const double dx = mimg(b.X[0] - a.X[0], lat.nx), dy = mimg(b.X[1] - a.X[1], lat.ny),
                   dz = mimg(b.X[2] - a.X[2], lat.nz);
      const int* bb = mbox + MBOX_N * a.nbl[k];
      const double lim = ra + sqrt((double)__int_as_float(bb[MBOX_R2])) + rc + 1.0;
      if (dx * dx + dy * dy + dz * dz > lim * lim) continue;
      bool boxes = true;
      for (int d = 0; d < 3 && boxes; ++d) {
        if (ba[d] > ba[3 + d] || bb[d] > bb[3 + d]) {  // an empty box: no members
          boxes = false;
          break;
        }
        // centres and half-lengths (in half cells) of the two boxes in lattice coordinates
        const int ca2 = 2 * a.o[d] + ba[d] + ba[3 + d], cb2 = 2 * b.o[d] + bb[d] + bb[3 + d];
        const int ha2 = ba[3 + d] - ba[d], hb2 = bb[3 + d] - bb[d];
        int sep2 = wrapi(cb2 - ca2, 2 * nn[d]);
        if (sep2 > nn[d]) sep2 = 2 * nn[d] - sep2;  // periodic distance of the centres
        if (sep2 - ha2 - hb2 > 2 * Rc) boxes = false;
      }
      nearby = boxes;
    }
    s_near = nearby;
  }
  __syncthreads();
  if (!s_near) return;
  const long long tb = dbits(thr);
  // grid-stride over the tile: a grid of a few waves, so that the common case (no pair in range,
  // every block leaves after the cull above) costs one short launch
  for (long long base = (long long)blockIdx.x * blockDim.x; base < a.sz; base += (long long)gridDim.x * blockDim.x) {
    const long long t = base + threadIdx.x;
    double F[3] = {0, 0, 0};
    bool has = false;
    TileCell c;
    if (t < a.sz && dbits(arena[a.off + t]) >= tb) {
      c = tile_cell(a, t, lat);
      const int g[3] = {c.gx, c.gy, c.gz};
      const int nn[3] = {lat.nx, lat.ny, lat.nz};
      for (int k = 0; k < a.nnb; ++k) {
        const BodyDev& b = bodies[a.nbl[k]];
        // this point's coordinates in the other body's tile, wrapped to [0, n); skip unless the point
        // lies within rc of that tile
        // tile coordinates of the other body's member cells (phi >= thr) lie in its box mbox (built by
        // the refill pass after the last flag update); the offsets reach Rc cells per axis, so a point
        // outside the box grown by Rc (periodically) finds no partner
        const int* bx = mbox + MBOX_N * a.nbl[k];
        int l[3];
        bool near = true;
        for (int d = 0; d < 3; ++d) {
          l[d] = wrapi_near(g[d] - b.o[d], nn[d]);
          const int lo = bx[d] - Rc, hi = bx[3 + d] + Rc;
          const bool in = (l[d] >= lo && l[d] <= hi) || (l[d] - nn[d] >= lo && l[d] - nn[d] <= hi) ||
                          (l[d] + nn[d] >= lo && l[d] + nn[d] <= hi);
          if (bx[d] > bx[3 + d] || !in) near = false;  // an empty box has no members
        }
        if (!near) continue;
        {
          // and within B's member radius (plus rc and a cell) of B's centre
          float dx = (float)c.gx - b.Xf[0], dy = (float)c.gy - b.Xf[1], dz = (float)c.gz - b.Xf[2];
          dx -= (float)lat.nx * rintf(dx / (float)lat.nx);
          dy -= (float)lat.ny * rintf(dy / (float)lat.ny);
          dz -= (float)lat.nz * rintf(dz / (float)lat.nz);
          const float lim = sqrtf(__int_as_float(bx[MBOX_R2])) + (float)rc + 1.0f;
          if (dx * dx + dy * dy + dz * dz > lim * lim) continue;
        }
        const double* bb = arena + b.off;
        // offsets in groups of 8: the group's loads are issued before any of them is tested (a
        // test per load would wait for each load in turn); contributions are added in offset order
        for (int j0 = 0; j0 < c_noff; j0 += 8) {
          double v[8];
  #pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int j = j0 + u;
            long long q = -1;
            if (j < c_noff) {
              int m[3];
              bool in = true;
              for (int d = 0; d < 3; ++d) {
                m[d] = l[d] + c_off[3 * j + d];  // |offset| <= 6: at most two wraps on a 4-cell side
                while (m[d] < 0) m[d] += nn[d];
                while (m[d] >= nn[d]) m[d] -= nn[d];
                in &= m[d] < b.L[d];
              }
              if (in) q = (long long)m[0] + (long long)b.L[0] * ((long long)m[1] + (long long)b.L[1] * m[2]);
            }
            v[u] = q >= 0 ? __ldg(bb + q) : 0.0;
          }
  #pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int j = j0 + u;
            if (j >= c_noff || dbits(v[u]) < tb) continue;
            F[0] += c_offf[3 * j];
            F[1] += c_offf[3 * j + 1];
            F[2] += c_offf[3 * j + 2];
            has = true;
          }
        }
      }
    }
    if (__ballot_sync(0xffffffffu, has) == 0) continue;
    double T[3] = {0, 0, 0};
    if (has) {
      const double arm[3] = {mimg(c.gx - a.X[0], lat.nx), mimg(c.gy - a.X[1], lat.ny), mimg(c.gz - a.X[2], lat.nz)};
      xcross(arm, F, T);
    }
    for (int p = 0; p < 3; ++p) {
      double sf = dwarp_sum(F[p]), st = dwarp_sum(T[p]);
      if ((threadIdx.x & 31) == 0) {
        if (sf != 0.0) atomicAdd(acc + (size_t)self * ACC_N + ACC_REP_F + p, sf);
        if (st != 0.0) atomicAdd(acc + (size_t)self * ACC_N + ACC_REP_T + p, st);
      }
    }
  }
}

// ---- rigid bodies ------------------------------------------------------------------------------
// Semi-implicit Euler with dt = 1: V += F/M, X += V, omega += I_w^-1 T with I_w = R I_body R^T,
// q <- normalize(exp(omega/2) q); fixed bodies keep V = omega = 0.
// A body whose update is not finite, or moves it by a lattice length or more in one step (a run
// that has blown up), is held at its last pose from then on and E_UNSTABLE is raised: every later
// kernel that derives a tile origin or a wrap from X gets finite, in-range values.
__device__ void integrate(BodyDev& b, const double* parts, const Lat& lat, StepState* st) {
  // FP64 throughout (GB300 issues FP64 at 1/64 of the FP32 rate and one thread runs this chain, so
  // the operation count is kept small: one reciprocal of M and of |q|, sincos, and the world-frame
  // inverse inertia applied as R (I_body^-1 (R^T T)) instead of being formed)
  double F[3], T[3];
  for (int a = 0; a < 3; ++a) {
    F[a] = parts[ACC_MOM_F + a] + parts[ACC_ADH_F + a] + parts[ACC_REP_F + a];
    T[a] = parts[ACC_MOM_T + a] + parts[ACC_ADH_T + a] + parts[ACC_REP_T + a];
    b.Xprev[a] = b.X[a];
  }
  if (b.fixed) {
    for (int a = 0; a < 3; ++a) {
      b.V[a] = 0;
      b.W[a] = 0;
    }
    return;
  }
  const int n[3] = {lat.nx, lat.ny, lat.nz};
  const double iM = 1.0 / b.M;
  const double Q0[4] = {b.Q[0], b.Q[1], b.Q[2], b.Q[3]};
  bool bad = false;
  for (int a = 0; a < 3; ++a) {
    b.V[a] += F[a] * iM;
    // finite and shorter than the lattice side (NaN fails the comparison)
    bad |= !(fabs(b.V[a]) < (double)n[a]);
    // periodic wrap in closed form (a move of less than a lattice side: the value of fmod)
    b.X[a] = wrapd(b.X[a] + b.V[a], n[a]);
  }
  double R[9];
  quat_R(b.Q, R);
  double t1[3], t2[3];
  for (int k = 0; k < 3; ++k) t1[k] = R[k] * T[0] + R[3 + k] * T[1] + R[6 + k] * T[2];  // R^T T
  for (int k = 0; k < 3; ++k) t2[k] = b.Ibinv[3 * k] * t1[0] + b.Ibinv[3 * k + 1] * t1[1] + b.Ibinv[3 * k + 2] * t1[2];
  for (int a = 0; a < 3; ++a) b.W[a] += R[3 * a] * t2[0] + R[3 * a + 1] * t2[1] + R[3 * a + 2] * t2[2];
  for (int a = 0; a < 3; ++a)
    if (b.rot_lock >> a & 1) b.W[a] = 0.0;
  const double wn = sqrt(b.W[0] * b.W[0] + b.W[1] * b.W[1] + b.W[2] * b.W[2]);
  if (wn > 0) {
    double sn, cs;
    sincos(0.5 * wn, &sn, &cs);
    const double s = sn / wn;
    const double dq[4] = {cs, b.W[0] * s, b.W[1] * s, b.W[2] * s};
    const double* q = b.Q;
    double nq[4] = {dq[0] * q[0] - dq[1] * q[1] - dq[2] * q[2] - dq[3] * q[3],
                    dq[0] * q[1] + dq[1] * q[0] + dq[2] * q[3] - dq[3] * q[2],
                    dq[0] * q[2] - dq[1] * q[3] + dq[2] * q[0] + dq[3] * q[1],
                    dq[0] * q[3] + dq[1] * q[2] - dq[2] * q[1] + dq[3] * q[0]};
    const double iq = 1.0 / sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
    for (int a = 0; a < 4; ++a) b.Q[a] = nq[a] * iq;
  }
  for (int a = 0; a < 3; ++a) bad |= !isfinite(b.W[a]) || !isfinite(b.X[a]);
  for (int a = 0; a < 4; ++a) bad |= !isfinite(b.Q[a]);
  if (bad) {
    for (int a = 0; a < 3; ++a) {
      b.X[a] = b.Xprev[a];
      b.V[a] = 0.0;
      b.W[a] = 0.0;
    }
    for (int a = 0; a < 4; ++a) b.Q[a] = Q0[a];
    b.fixed = 1;
    atomicOr(&st->err, E_UNSTABLE);
  }
}

__global__ void __launch_bounds__(256) k_bodies(BodyDev* bodies, int nb, double* acc, double* last, double* volacc,
                                                StepState* st, Lat lat, double* rtab, int Lmax, int* mbox,
                                                double* fsum) {
  const int n[3] = {lat.nx, lat.ny, lat.nz};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    BodyDev& b = bodies[i];
    double* a = acc + (size_t)i * ACC_N;
    integrate(b, a, lat, st);
    mirror_f(b);
    // running sums of the total force and torque (mean forces over many steps without host reads)
    for (int c = 0; c < 3; ++c) {
      fsum[6 * i + c] += a[ACC_MOM_F + c] + a[ACC_ADH_F + c] + a[ACC_REP_F + c];
      fsum[6 * i + 3 + c] += a[ACC_MOM_T + c] + a[ACC_ADH_T + c] + a[ACC_REP_T + c];
    }
    for (int k = 0; k < ACC_N; ++k) {
      last[(size_t)i * ACC_N + k] = a[k];
      a[k] = 0.0;
    }
    volacc[2 * i] = 0.0;
    volacc[2 * i + 1] = 0.0;
    for (int a = 0; a < 3; ++a) {  // member record: rebuilt by this step's refill pass
      mbox[MBOX_N * i + a] = INT_MAX;
      mbox[MBOX_N * i + 3 + a] = INT_MIN;
    }
    mbox[MBOX_N * i + MBOX_R2] = 0;
    for (int d = 0; d < 3; ++d) {
      b.o_prev[d] = b.o[d];
      if (b.L[d] < n[d]) b.o[d] = (int)floor(b.X[d] + 0.5) - b.L[d] / 2;
    }
  }
  __syncthreads();
  // per body and axis, the minimum-image offset of every tile coordinate from the pre-update centre
  // (the advection's face velocities need it; the table saves each cell the FP64 wrap)
  for (int k = threadIdx.x; k < nb * 3 * Lmax; k += blockDim.x) {
    const int i = k / (3 * Lmax), a = (k / Lmax) % 3, l = k % Lmax;
    const BodyDev& b = bodies[i];
    if (l < b.L[a]) rtab[k] = mimg(wrapi_near(b.o[a] + l, n[a]) - b.Xprev[a], n[a]);
  }
  build_lists(bodies, nb, lat, st);
  if (threadIdx.x == 0) {
    st->nbnd = 0;    // the boundary list is rebuilt by the refill pass after the new flags
    st->ncover = 0;  // counted by the flag pass
  }
}

// End of a step: the fluid mass (fixed-order sum of the collision's per-block partials, which are
// cleared) and the population buffer flip. The bulk collision may run beside the body update, so
// neither can happen earlier.
__global__ void __launch_bounds__(256) k_finish(double* mass_part, unsigned n_mass_part, StepState* st) {
  __shared__ double red[256];
  double sm = 0.0;
  for (unsigned k = threadIdx.x; k < n_mass_part; k += blockDim.x) {
    sm += mass_part[k];
    mass_part[k] = 0.0;
  }
  red[threadIdx.x] = sm;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->last_mass = red[0];
    st->parity ^= 1;
    st->psi_skip = 0;
  }
}

// ---- advection ---------------------------------------------------------------------------------
// Monotonized-central slope: 0 unless dm and dp have the same sign, else
// sign(dm) min(2|dm|, |dm + dp| / 2, 2|dp|). Evaluated on bit patterns, with the same result as the
// plain FP64 form: doubling and halving a normal double add to or subtract from its exponent field,
// and non-negative doubles order like their bit patterns. Only dm + dp is an FP64 operation (GB300
// issues FP64 at 1/64 of the FP32 rate). The differences of phase-field values that reach this
// function are 0 or far above the subnormal range, so no product underflows and no half is
// subnormal.
__device__ __forceinline__ double mc_slope(double dm, double dp) {
  const long long bm = dbits(dm), bp = dbits(dp);
  const long long mag = 0x7FFFFFFFFFFFFFFFLL, one_exp = 1LL << 52;
  const long long am = bm & mag, ap = bp & mag;
  if (((bm ^ bp) < 0) || am == 0 || ap == 0) return 0.0;
  const long long two_am = am + one_exp, two_ap = ap + one_exp;
  const long long half_s = (dbits(dm + dp) & mag) - one_exp;
  long long m = two_am < half_s ? two_am : half_s;
  m = m < two_ap ? m : two_ap;
  return __longlong_as_double(m | (bm & (long long)0x8000000000000000ULL));
}

// one sweep along axis d: out (origin b.o) <- in (origin o_in). The x-sweep reads with the previous
// origin, so the recentring shift (at most one cell per axis and step) is folded into it. Stencil
// values are addressed in tile-local coordinates; a periodic axis (tile as long as the lattice)
// wraps, any other axis reads zero outside the tile.
__device__ __forceinline__ int in_local(int i, int shift, int L, int n) {
  int l = i + shift;
  if (L == n) l = l < 0 ? l + n : (l >= n ? l - n : l);
  return l;
}

__global__ void __launch_bounds__(256) k_sweep(const BodyDev* bodies, double* arena, Lat lat, int d, int in_buf,
                                               int out_buf, int use_prev, int last, double* volacc, StepState* st,
                                               const double* __restrict__ rtab, int Lmax) {
  // The cells whose stencil is not flat (the interface shell) are gathered into the first lanes of
  // the block before the flux arithmetic: GB300 issues FP64 at 1/64 of the FP32 rate and a warp
  // instruction occupies the FP64 pipe for all its lanes, active or not, so scattered interface
  // cells left most of its time idle. The arithmetic per cell is unchanged.
  __shared__ double cp[5][256];
  __shared__ double cr[2][256];
  __shared__ double cv[256];
  __shared__ int ncomp;
  const int self = blockIdx.y;
  const BodyDev& b = bodies[self];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (threadIdx.x == 0) ncomp = 0;
  __syncthreads();
  double v = 0.0;
  const bool inside = t < b.sz;
  bool nonflat = false;
  double p[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, r1 = 0.0, r2 = 0.0;
  const int nn[3] = {lat.nx, lat.ny, lat.nz};
  int ii[3] = {0, 0, 0};
  if (inside) {
    {
      const unsigned u = (unsigned)t, L0 = (unsigned)b.L[0], L1 = (unsigned)b.L[1];
      const unsigned r = u / L0;
      ii[0] = (int)(u - r * L0);
      ii[1] = (int)(r % L1);
      ii[2] = (int)(r / L1);
    }
    // input-local coordinates of this output cell
    int li[3];
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      // origins are unwrapped integers: take the shift as the minimum image of their difference
      int shift = 0;
      if (use_prev && b.L[a] < nn[a]) {
        shift = wrapi_near(b.o[a] - b.o_prev[a], nn[a]);
        if (shift > nn[a] / 2) shift -= nn[a];
      }
      li[a] = in_local(ii[a], shift, b.L[a], nn[a]);
      if (a != d && (li[a] < 0 || li[a] >= b.L[a])) ok = false;
    }
    const double* in = arena + b.off + (long long)in_buf * b.sz;
    const long long sd = d == 0 ? 1 : (d == 1 ? (long long)b.L[0] : (long long)b.L[0] * b.L[1]);
    const long long base = li[0] + (long long)b.L[0] * (li[1] + (long long)b.L[1] * li[2]) - (long long)li[d] * sd;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const int l = in_local(li[d], k - 2, b.L[d], b.L[d] == nn[d] ? nn[d] : -1);
      p[k] = (ok && l >= 0 && l < b.L[d]) ? in[base + l * sd] : 0.0;
    }
    const long long b2 = dbits(p[2]);
    // flat stencil: both face fluxes are u * p with the same u, so the update is exactly zero
    v = p[2];
    nonflat = !(dbits(p[0]) == b2 && dbits(p[1]) == b2 && dbits(p[3]) == b2 && dbits(p[4]) == b2);
    if (nonflat) {
      // the face velocity u_d (the d-component of V + omega x r, r about X_prev) depends only on the
      // two other coordinates, so both faces of the cell share it;
      // r_a = mimg(wrap(o_a + i_a) - Xprev_a) from the per-body table built by k_bodies
      const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
      const double* rt = rtab + (size_t)self * 3 * Lmax;
      r1 = rt[d1 * Lmax + ii[d1]];
      r2 = rt[d2 * Lmax + ii[d2]];
    }
  }
  int slot = -1;
  {
    const unsigned m = __ballot_sync(0xffffffffu, nonflat);
    if (m) {
      const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(&ncomp, __popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (nonflat) {
        slot = base + __popc(m & ((1u << lane) - 1u));
#pragma unroll
        for (int k = 0; k < 5; ++k) cp[k][slot] = p[k];
        cr[0][slot] = r1;
        cr[1][slot] = r2;
      }
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < ncomp) {
    const int c = threadIdx.x;
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    double q[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) q[k] = cp[k][c];
    const double u = b.V[d] + (b.W[d1] * cr[1][c] - b.W[d2] * cr[0][c]);
    double Fl, Fr;
    {
      const double face = u >= 0.0 ? q[1] + 0.5 * (1.0 - u) * mc_slope(q[1] - q[0], q[2] - q[1])
                                   : q[2] - 0.5 * (1.0 + u) * mc_slope(q[2] - q[1], q[3] - q[2]);
      Fl = u * face;
    }
    {
      const double face = u >= 0.0 ? q[2] + 0.5 * (1.0 - u) * mc_slope(q[2] - q[1], q[3] - q[2])
                                   : q[3] - 0.5 * (1.0 + u) * mc_slope(q[3] - q[2], q[4] - q[3]);
      Fr = u * face;
    }
    cv[c] = q[2] - (Fr - Fl);
  }
  __syncthreads();
  if (slot >= 0) v = cv[slot];
  if (inside) {
    arena[b.off + (long long)out_buf * b.sz + t] = v;
    if (last && (dbits(v) << 1) > (dbits(PHI_EPS) << 1)) {  // |v| > PHI_EPS
      // the outer two layers must stay empty (they are the stencil halo); a moving body's upwind
      // scheme leaves a geometrically decaying tail ahead of its front, and the tile drops what
      // reaches past it, so values of at most PHI_EPS there are tolerated
      bool edge = false;
      for (int a = 0; a < 3; ++a)
        if (b.L[a] < nn[a] && (ii[a] < 2 || ii[a] >= b.L[a] - 2)) edge = true;
      if (edge) atomicOr(&st->err, E_TILE);
    }
  }
  if (last) {
    // volume (sum phi) and interface-cell count of the body: warp sums, then one FP64 atomic per
    // block (per-warp atomics on the same two words would queue up)
    __shared__ double wv[8];
    __shared__ int wc[8];
    const long long vb = dbits(v);
    const bool live = inside && (vb << 1) != 0;
    double sv = 0.0;
    int cnt = 0;
    if (__ballot_sync(0xffffffffu, live)) {
      sv = dwarp_sum(live ? v : 0.0);
      const bool in_if = live && vb > dbits(PHI_EPS) && vb < dbits(1.0 - PHI_EPS);
      cnt = __popc(__ballot_sync(0xffffffffu, in_if));
    }
    if ((threadIdx.x & 31) == 0) {
      wv[threadIdx.x >> 5] = sv;
      wc[threadIdx.x >> 5] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bv = 0.0;
      int bc = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        bv += wv[w];
        bc += wc[w];
      }
      if (bv != 0.0) atomicAdd(volacc + 2 * self, bv);
      if (bc != 0) atomicAdd(volacc + 2 * self + 1, (double)bc);
    }
  }
}

__global__ void k_volume(const BodyDev* bodies, const double* arena, double* volacc) {
  const int self = blockIdx.y;
  const BodyDev& b = bodies[self];
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = t < b.sz ? arena[b.off + t] : 0.0;
  double sv = dwarp_sum(v);
  double sc = dwarp_sum((v > PHI_EPS && v < 1.0 - PHI_EPS) ? 1.0 : 0.0);
  if ((threadIdx.x & 31) == 0) {
    if (sv != 0.0) atomicAdd(volacc + 2 * self, sv);
    if (sc != 0.0) atomicAdd(volacc + 2 * self + 1, sc);
  }
}

// ---- MPF kinetics ------------------------------------------------------------------------------
// For body a at cell g: active phases = solids with phi > PHI_EPS at g or a face neighbour, plus the
// fluid if 1 - sum phi > PHI_EPS there; N = their number; explicit Euler step of
// phi_a += sum_b (M/N) [ s_ab (I_a - I_b) + sum_c (s_bc - s_ac) I_c + (D_a - D_b if 0<phi_a<1) ]
// with I = lap(phi) + (pi/eta)^2 phi, D_B = (V_B(0) - sum phi_B) / #{0 < phi_B < 1}, D_fluid = 0.
constexpr int MAXACT = 8;

// Kinetics constants evaluated once on the host with the same expressions the kernel used per cell
// (IEEE division is correctly rounded on both sides, so the values are identical): pi^2 / eta^2 and
// M / N for every possible number of active phases N (an FP64 division costs many FP64-pipe
// instructions, and GB300 issues FP64 at 1/64 of the FP32 rate).
struct KinParams {
  double k2, s_sf, s_ss;
  double mobN[MAXACT + 2];
};

// phi at a cell of a tile given in tile-local coordinates l and its 6 face neighbours (order: self,
// +x, -x, +y, -y, +z, -z); periodic tile axes wrap, other axes read zero outside the tile
__device__ __forceinline__ void tile_val7(const double* buf, const int L[3], const int l[3], const int nn[3],
                                          double out[7]) {
  const long long s1 = L[0], s2 = (long long)L[0] * L[1];
  const bool in0 = l[0] >= 0 && l[0] < L[0] && l[1] >= 0 && l[1] < L[1] && l[2] >= 0 && l[2] < L[2];
  const long long c = l[0] + s1 * l[1] + s2 * l[2];
  out[0] = in0 ? buf[c] : 0.0;
  const long long st[3] = {1, s1, s2};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
      const int dlt = sg == 0 ? 1 : -1;
      int q[3] = {l[0], l[1], l[2]};
      q[a] += dlt;
      if (L[a] == nn[a]) q[a] = q[a] < 0 ? q[a] + nn[a] : (q[a] >= nn[a] ? q[a] - nn[a] : q[a]);
      const bool ok = q[0] >= 0 && q[0] < L[0] && q[1] >= 0 && q[1] < L[1] && q[2] >= 0 && q[2] < L[2];
      out[1 + 2 * a + sg] = ok ? buf[q[0] + s1 * q[1] + s2 * q[2]] : 0.0;
      (void)st;
    }
  }
}

__global__ void __launch_bounds__(256) k_kinetics(const BodyDev* bodies, double* arena, const double* volacc, Lat lat,
                                                  KinParams kp) {
  const int self = blockIdx.y;
  const BodyDev& b = bodies[self];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // volume-restoring term D of this body (slot 0) and of each listed neighbour (slot k + 1), once per
  // block: D = (V(0) - sum phi) / #{0 < phi < 1}, 0 without interface cells
  __shared__ double sD[MAXNB + 1];
  for (int k = threadIdx.x; k <= b.nnb; k += blockDim.x) {
    const int id = k == 0 ? self : b.nbl[k - 1];
    const double cnt = volacc[2 * id + 1];
    sD[k] = cnt > 0.0 ? (bodies[id].vol_ref - volacc[2 * id]) / cnt : 0.0;
  }
  __syncthreads();
  if (t >= b.sz) return;
  const double* in = arena + b.off + b.sz;  // buffer 1: advected field
  double* out = arena + b.off;              // buffer 0: new field
  const int nn[3] = {lat.nx, lat.ny, lat.nz};
  int ii[3];
  {
    const unsigned u = (unsigned)t, L0 = (unsigned)b.L[0], L1 = (unsigned)b.L[1];
    const unsigned r = u / L0;
    ii[0] = (int)(u - r * L0);
    ii[1] = (int)(r % L1);
    ii[2] = (int)(r / L1);
  }
  double pa[7];
  tile_val7(in, b.L, ii, nn, pa);
  const long long eb = dbits(PHI_EPS);
  bool act_a = false;
#pragma unroll
  for (int k = 0; k < 7; ++k) act_a |= dbits(pa[k]) > eb;
  if (!act_a) {
    out[t] = pa[0];
    return;
  }
  const int g[3] = {wrapi_near(b.o[0] + ii[0], nn[0]), wrapi_near(b.o[1] + ii[1], nn[1]),
                    wrapi_near(b.o[2] + ii[2], nn[2])};
  // is any other body present in this cell's 7-point stencil?
  bool others = false;
  for (int k = 0; k < b.nnb && !others; ++k) {
    const BodyDev& o = bodies[b.nbl[k]];
    int lo[3];
    bool near = true;
    for (int a = 0; a < 3; ++a) {
      lo[a] = wrapi_near(g[a] - o.o[a], nn[a]);
      if (o.L[a] < nn[a]) {
        if (lo[a] > nn[a] - 2) lo[a] -= nn[a];
        if (lo[a] < -1 || lo[a] > o.L[a]) near = false;
      }
    }
    if (!near) continue;
    double v7[7];
    tile_val7(arena + o.off + o.sz, o.L, lo, nn, v7);
    for (int k2 = 0; k2 < 7; ++k2) others |= dbits(v7[k2]) > eb;
  }
  if (!others) {
    // one solid phase a and the fluid f = 1 - phi: N = 2 where the fluid is present at the cell or a
    // face neighbour, and then the rate is (M/2) [sigma_sf (I_a - I_f) + D_a (interface cells)]. With
    // lap = the 7-point Laplacian of phi, I_a = lap + k2 phi and I_f = -lap + k2 (1 - phi), so
    // I_a - I_f = 2 lap + k2 (2 phi - 1) (the same quantity as the general form below, up to
    // rounding). Presence of the fluid (1 - phi > PHI_EPS) is tested on bit patterns.
    const long long one_eb = dbits(1.0 - PHI_EPS), neg0 = (long long)0x8000000000000000ULL;
    bool fl = false;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const long long bk = dbits(pa[k]);
      fl |= (bk == neg0 ? 0LL : bk) < one_eb;
    }
    if (!fl) {  // N = 1: no kinetics
      out[t] = pa[0];
      return;
    }
    double lap = 0.0;
#pragma unroll
    for (int k = 1; k < 7; ++k) lap += pa[k];
    lap -= 6.0 * pa[0];
    double term = kp.s_sf * (2.0 * lap + kp.k2 * (2.0 * pa[0] - 1.0));
    if (dbits(pa[0]) > eb && dbits(pa[0]) < one_eb) term += sD[0];
    out[t] = pa[0] + kp.mobN[2] * term;
    return;
  }
  // active solids in ascending id order, with their 7-point values
  double vals[MAXACT][7];
  int dslot[MAXACT];  // slot of each active phase in sD
  int na = 0;
  int pos_self = -1;
  double S[7] = {0, 0, 0, 0, 0, 0, 0};
  int k_nb = 0;
  for (int step = 0; step <= b.nnb; ++step) {
    int id;
    if (pos_self < 0 && (k_nb >= b.nnb || b.nbl[k_nb] > self)) id = self;
    else id = b.nbl[k_nb++];
    if (id == self) {
      pos_self = na;
      for (int k = 0; k < 7; ++k) {
        vals[na][k] = pa[k];
        S[k] += pa[k];
      }
      dslot[na] = 0;
      ++na;
      continue;
    }
    const int slot = k_nb;  // b.nbl[slot - 1] == id
    const BodyDev& o = bodies[id];
    int lo[3];
    bool near = true;
    for (int a = 0; a < 3; ++a) {
      lo[a] = wrapi_near(g[a] - o.o[a], nn[a]);
      if (o.L[a] < nn[a]) {
        if (lo[a] > nn[a] - 2) lo[a] -= nn[a];  // just below the tile: keep the +1 neighbour reachable
        if (lo[a] < -1 || lo[a] > o.L[a]) near = false;
      }
    }
    if (!near) continue;
    double v7[7];
    tile_val7(arena + o.off + o.sz, o.L, lo, nn, v7);
    bool on = false;
    for (int k = 0; k < 7; ++k) on |= dbits(v7[k]) > eb;
    if (!on) continue;
    if (na < MAXACT - (pos_self < 0 ? 1 : 0)) {  // always keep a slot for self
      for (int k = 0; k < 7; ++k) {
        vals[na][k] = v7[k];
        S[k] += v7[k];
      }
      dslot[na] = slot;
      ++na;
    }
  }
  // S >= 0, so the signed bit patterns order like the values
  const long long one_eb = dbits(1.0 - PHI_EPS);
  bool fl = false;
  for (int k = 0; k < 7; ++k) fl |= dbits(S[k]) < one_eb;
  const int N = na + (fl ? 1 : 0);
  if (N <= 1) {
    out[t] = pa[0];
    return;
  }
  const double k2 = kp.k2;
  double I[MAXACT + 1], D[MAXACT + 1];
  for (int j = 0; j < na; ++j) {
    double lap = 0.0;
    for (int k = 1; k < 7; ++k) lap += vals[j][k];
    lap -= 6.0 * vals[j][0];
    I[j] = lap + k2 * vals[j][0];
    D[j] = sD[dslot[j]];
  }
  if (fl) {
    double lap = 0.0;
    for (int k = 1; k < 7; ++k) lap += 1.0 - S[k];
    lap -= 6.0 * (1.0 - S[0]);
    I[na] = lap + k2 * (1.0 - S[0]);
    D[na] = 0.0;
  }
  const double s_sf = kp.s_sf, s_ss = kp.s_ss;
  auto sig = [&](int p, int q) { return (p == na || q == na) ? s_sf : s_ss; };
  const int a = pos_self;
  const bool in_if = dbits(pa[0]) > eb && dbits(pa[0]) < one_eb;
  double rate = 0.0;
  for (int bq = 0; bq < N; ++bq) {
    if (bq == a) continue;
    double term = sig(a, bq) * (I[a] - I[bq]);
    for (int gg = 0; gg < N; ++gg) {
      if (gg == a || gg == bq) continue;
      term += (sig(bq, gg) - sig(a, gg)) * I[gg];
    }
    if (in_if) term += D[a] - D[bq];
    rate += kp.mobN[N] * term;
  }
  out[t] = pa[0] + rate;
}

// ---- dense read-out ----------------------------------------------------------------------------
__global__ void k_fill(double* out, long long N, double v) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N) out[n] = v;
}

// body >= 0: scatter that body's field; body < 0: 1 - sum of all bodies (fluid phase)
__global__ void k_phi_scatter(const BodyDev* bodies, const double* arena, double* out, Lat lat, int body) {
  const int self = body >= 0 ? body : blockIdx.y;
  const BodyDev& b = bodies[self];
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b.sz) return;
  TileCell c = tile_cell(b, t, lat);
  const long long n = c.gx + (long long)lat.nx * (c.gy + (long long)lat.ny * c.gz);
  if (body >= 0) {
    out[n] = arena[b.off + t];
    return;
  }
  if (b.nnb && covered_by_lower_body(bodies, b, self, c.gx, c.gy, c.gz, lat)) return;
  double S = arena[b.off + t];
  for (int k = 0; k < b.nnb; ++k) {
    const BodyDev& o = bodies[b.nbl[k]];
    if (b.nbl[k] < self) continue;
    long long j = tile_index(o.o, o.L, c.gx, c.gy, c.gz, lat);
    if (j >= 0) S += arena[o.off + j];
  }
  out[n] = 1.0 - S;
}

// before the bodies are moved: every cell of their current tiles loses its flags, except that a
// solid cell keeps the solid bit under the owner id F_STALE, so the next flag pass does not count
// it as covered again
__global__ void k_clear_tile_flags(const BodyDev* bodies, uint16_t* flags, Lat lat) {
  const BodyDev& b = bodies[blockIdx.y];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b.sz) return;
  const TileCell c = tile_cell(b, t, lat);
  uint16_t& f = flags[c.gx + (long long)lat.nx * (c.gy + (long long)lat.ny * c.gz)];
  f = (f & F_SOLID) ? (uint16_t)(F_SOLID | F_STALE) : (uint16_t)0;
}

// after the flag pass at the new poses: cells still marked stale lie outside every new tile and
// are uncovered (their populations were zeroed while they were solid)
__global__ void k_clear_stale(uint16_t* flags, long long N) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < N && flags[n] == (uint16_t)(F_SOLID | F_STALE)) flags[n] = 0;
}

// ---- launchers ---------------------------------------------------------------------------------
static dim3 tile_grid(int max_tile, int nb) { return dim3((unsigned)((max_tile + 255) / 256), (unsigned)nb); }

void launch_rasterize(const Lat& lat, BodyDev* bodies, int nb, int max_tile, double* arena, double eta,
                      cudaStream_t s) {
  if (nb) k_rasterize<<<tile_grid(max_tile, nb), 256, 0, s>>>(bodies, arena, lat, eta);
}
void launch_neighbour_lists(BodyDev* bodies, int nb, const Lat& lat, StepState* st, cudaStream_t s) {
  if (nb) k_neighbour_lists<<<1, 256, 0, s>>>(bodies, nb, lat, st);
}
void launch_flags(const Lat& lat, BodyDev* bodies, int nb, int max_tile, double* arena, uint16_t* flags,
                  double threshold, int init, StepState* st, cudaStream_t s) {
  if (nb) k_flags<<<tile_grid(max_tile, nb), 256, 0, s>>>(bodies, arena, flags, lat, threshold, init, st);
}
void launch_body_props(const Lat& lat, BodyDev* bodies, int nb, int max_tile, double* arena, double* scratch,
                       cudaStream_t s) {
  if (!nb) return;
  cudaMemsetAsync(scratch, 0, sizeof(double) * 9 * nb, s);
  k_body_props<<<tile_grid(max_tile, nb), 256, 0, s>>>(bodies, arena, scratch, lat, 0);
  k_body_props_finish<<<(nb + 127) / 128, 128, 0, s>>>(bodies, nb, scratch, lat, 0);
  cudaMemsetAsync(scratch, 0, sizeof(double) * 9 * nb, s);
  k_body_props<<<tile_grid(max_tile, nb), 256, 0, s>>>(bodies, arena, scratch, lat, 1);
  k_body_props_finish<<<(nb + 127) / 128, 128, 0, s>>>(bodies, nb, scratch, lat, 1);
}
void launch_repulsion(const Lat& lat, const BodyDev* bodies, int nb, int max_tile, const double* arena, double* acc,
                      const PhysParams& pp, const int* mbox, cudaStream_t s) {
  if (nb > 1 && pp.e0 != 0.0) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    dim3 g = tile_grid(max_tile, nb);
    // a few waves in all, but never more than four chunks of the tile per block (many bodies)
    const unsigned cap = std::max((g.x + 3) / 4, (unsigned)std::max(1, 4 * nsm / (nb * g_launch_share)));
    if (g.x > cap) g.x = cap;
    k_repulsion<<<g, 256, 0, s>>>(bodies, arena, acc, lat, pp.rc, (int)std::ceil(pp.rc), pp.member_threshold, pp.eta,
                                  mbox);
  }
}
void launch_bodies(const Lat& lat, BodyDev* bodies, int nb, double* acc, double* last, double* volacc,
                   StepState* st, double* rtab, int Lmax, int* mbox, double* fsum, cudaStream_t s) {
  if (nb) k_bodies<<<1, 256, 0, s>>>(bodies, nb, acc, last, volacc, st, lat, rtab, Lmax, mbox, fsum);
}
void launch_finish(double* mass_part, unsigned n_mass_part, StepState* st, cudaStream_t s) {
  k_finish<<<1, 256, 0, s>>>(mass_part, n_mass_part, st);
}
void launch_advect(const Lat& lat, const BodyDev* bodies, int nb, int max_tile, double* arena, int mpf, double* volacc,
                   StepState* st, const double* rtab, int Lmax, cudaStream_t s) {
  if (!nb) return;
  dim3 g = tile_grid(max_tile, nb);
  k_sweep<<<g, 256, 0, s>>>(bodies, arena, lat, 0, 0, 1, 1, 0, volacc, st, rtab, Lmax);
  k_sweep<<<g, 256, 0, s>>>(bodies, arena, lat, 1, 1, 2, 0, 0, volacc, st, rtab, Lmax);
  k_sweep<<<g, 256, 0, s>>>(bodies, arena, lat, 2, 2, mpf ? 1 : 0, 0, 1, volacc, st, rtab, Lmax);
}
void launch_kinetics(const Lat& lat, const BodyDev* bodies, int nb, int max_tile, double* arena, const double* volacc,
                     const PhysParams& pp, cudaStream_t s) {
  if (!nb) return;
  KinParams kp;
  kp.k2 = PI * PI / (pp.eta * pp.eta);
  kp.s_sf = pp.sigma_sf;
  kp.s_ss = pp.sigma_ss;
  for (int k = 0; k < MAXACT + 2; ++k) kp.mobN[k] = k ? pp.mobility / k : 0.0;
  k_kinetics<<<tile_grid(max_tile, nb), 256, 0, s>>>(bodies, arena, volacc, lat, kp);
}
void launch_phi_dense(const Lat& lat, const BodyDev* bodies, int nb, int max_tile, const double* arena, int body,
                      double* out, cudaStream_t s) {
  k_fill<<<(unsigned)((lat.N + 255) / 256), 256, 0, s>>>(out, lat.N, body >= 0 ? 0.0 : 1.0);
  if (!nb) return;
  dim3 g = tile_grid(max_tile, body >= 0 ? 1 : nb);
  k_phi_scatter<<<g, 256, 0, s>>>(bodies, arena, out, lat, body);
}

void launch_clear_tile_flags(const Lat& lat, const BodyDev* bodies, int nb, int max_tile, uint16_t* flags,
                             cudaStream_t s) {
  if (nb) k_clear_tile_flags<<<tile_grid(max_tile, nb), 256, 0, s>>>(bodies, flags, lat);
}
__global__ void k_reset_member_boxes(int* mbox, int nb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < MBOX_N * nb) {
    const int e = k % MBOX_N;
    mbox[k] = e < 3 ? INT_MAX : (e < 6 ? INT_MIN : 0);
  }
}
void launch_reset_member_boxes(int* mbox, int nb, cudaStream_t s) {
  if (nb) k_reset_member_boxes<<<(MBOX_N * nb + 255) / 256, 256, 0, s>>>(mbox, nb);
}
void launch_clear_stale(const Lat& lat, uint16_t* flags, cudaStream_t s) {
  k_clear_stale<<<(unsigned)((lat.N + 255) / 256), 256, 0, s>>>(flags, lat.N);
}

}  // namespace cbl
