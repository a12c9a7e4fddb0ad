// Lattice-Boltzmann kernels of the capillary-bridge step (Sec. 3.2 of arXiv:1902.10432).
//
//  k_density  : pull streaming with half-way bounce-back, density, psi = 1 - exp(-rho/rho0)
//               (Eq. lb_streaming, Eq. lb_bounce_back, Eq. mean_field_potential); solid cells
//               carry psi of their owner's wetting density (Sec. 3.2.3).
//  k_collide  : Shan-Chen force (Eq. benzi_force), pull again, moving-wall term g and local mass
//               correction (Eqs. lb_bounce_back_us, lb_bounce_back_mass), Guo-forced BGK
//               collision (Eqs. lb_collision, distribution_eq, guo_forcing, fluid_velocity),
//               FP64 fluid-mass partial sums.
//  k_fused    : the two above in one pass over HBM (psi of each z-plane and a one-cell ring kept in
//               shared memory, populations pulled again for the collision from the caches); fluid
//               cells next to a solid are left to k_collide_near, fed by k_density_tiles.
//  k_collide_acc, k_psi_fixup : the collision that also sums the next step's density from the
//               values it stores (regions marched along z, shared-memory exchange), and the
//               completion of psi at the regions' edges at the start of the next step.
//  k_collide_near : the collision of the fluid cells next to a solid (the boundary-cell list).
//  k_boundary : over the same list: momentum exchange on the bodies (Eq. solid_liquid_force) and
//               the reaction of the Shan-Chen force (Sec. 3.2.3), summed in FP64.
//  k_batch_lbm : the density and bulk collision of every instance of a batch in one persistent
//               launch (work queue, bounded grid barrier).
//  k_refill   : cover refill of nodes that became solid (Sec. 3.2.2), as a gather over each
//               fluid node's 26 neighbours so that no two threads write the same populations; the
//               same scan rebuilds the boundary-cell list for the next step.
//
// Populations are SoA, f[i * N + n], in FP64, FP32 or binary16 deviations from the weights.
//
// This file is compiled once per velocity set: as itself for D3Q19 (namespace cbl::q19) and through
// lbm27.cu with CBL_Q = 27 (namespace cbl::q27). The no-allocation entry point exists for D3Q19
// only.
#include <algorithm>
#include <climits>
#include <cmath>
#include "../../include/cbl.h"
#include "cbl_dev.cuh"

#ifndef CBL_Q
#define CBL_Q 19
#endif

namespace cbl {
#if CBL_Q == 27
namespace q27 {
#elif CBL_Q == 19
namespace q19 {
#else
#error "CBL_Q must be 19 or 27"
#endif

__constant__ float c_wh[Q];  // binary16-rounded weights: base of the FP16-deviation storage

void set_fp16_weights(cudaStream_t s) {
  float wh[Q];
  for (int i = 0; i < Q; ++i) wh[i] = __half2float(__float2half_rn((float)w_of(i)));
  cudaMemcpyToSymbolAsync(c_wh, wh, sizeof(wh), 0, cudaMemcpyHostToDevice, s);
}

template <typename S>
struct St;
template <>
struct St<double> {
  using R = double;
  __device__ static R ld(const double* p, size_t k, int) { return __ldg(p + k); }
  __device__ static void st(double* p, size_t k, int, R v) { p[k] = v; }
  __device__ static R rt(R v, int) { return v; }
};
template <>
struct St<float> {
  using R = float;
  __device__ static R ld(const float* p, size_t k, int) { return __ldg(p + k); }
  __device__ static void st(float* p, size_t k, int, R v) { p[k] = v; }
  __device__ static R rt(R v, int) { return v; }
};
template <>
struct St<__half> {
  using R = float;
  // f = h + w_hat: zero populations (solid cells) are stored exactly as h = -w_hat.
  __device__ static R ld(const __half* p, size_t k, int i) { return __half2float(__ldg(p + k)) + c_wh[i]; }
  __device__ static R from_raw(unsigned short h, int i) { return __half2float(__ushort_as_half(h)) + c_wh[i]; }
  __device__ static void st(__half* p, size_t k, int i, R v) { p[k] = __float2half_rn(v - c_wh[i]); }
  // the value a later load of the stored population returns
  __device__ static R rt(R v, int i) { return __half2float(__float2half_rn(v - c_wh[i])) + c_wh[i]; }
};

// Density and pseudo-potential of a fluid cell next to a solid, as its collision used them; the
// solid-fluid force pass reads them back, so its g_i and psi are the collision's own.
template <typename R>
struct RhoPsi {
  R rho, psi;
};

// A lattice cell with its neighbour offsets: nbr(c, i, s) is the index of x + s c_i, built from
// per-axis offsets for -1, 0, +1 that already contain the periodic wrap (32-bit: the lattice holds
// fewer than 2^31 cells).
struct Cell {
  int x, y, z;
  unsigned n;
  int ox[3], oy[3], oz[3];
};

__device__ __forceinline__ Cell make_cell(int x, int y, int z, const Lat& lat) {
  Cell c;
  c.x = x;
  c.y = y;
  c.z = z;
  const int nx = lat.nx, nxy = lat.nx * lat.ny;
  c.n = (unsigned)x + (unsigned)nx * ((unsigned)y + (unsigned)lat.ny * (unsigned)z);
  c.ox[0] = x ? -1 : nx - 1;
  c.ox[1] = 0;
  c.ox[2] = x + 1 < nx ? 1 : -(nx - 1);
  c.oy[0] = y ? -nx : nx * (lat.ny - 1);
  c.oy[1] = 0;
  c.oy[2] = y + 1 < lat.ny ? nx : -nx * (lat.ny - 1);
  c.oz[0] = z ? -nxy : nxy * (lat.nz - 1);
  c.oz[1] = 0;
  c.oz[2] = z + 1 < lat.nz ? nxy : -nxy * (lat.nz - 1);
  return c;
}

__device__ __forceinline__ Cell cell_of(long long n, const Lat& lat) {
  const unsigned u = (unsigned)n, nx = (unsigned)lat.nx, ny = (unsigned)lat.ny;
  const unsigned r = u / nx;
  return make_cell((int)(u - r * nx), (int)(r % ny), (int)(r / ny), lat);
}

// neighbour x + s * c_i (s = +1 downstream, -1 upstream)
__device__ __forceinline__ long long nbr(const Cell& c, const Lat& lat, int i, int s) {
  (void)lat;
  return (long long)(c.n + (unsigned)(c.ox[1 + s * cx_of(i)] + c.oy[1 + s * cy_of(i)] + c.oz[1 + s * cz_of(i)]));
}

// Pull: f_i(x) = f*_i(x - c_i) from a fluid source, else f*_opp(i)(x) (half-way bounce-back).
// A cell without the near-solid flag has no solid neighbour, so its sources need no test.
template <typename S>
__device__ __forceinline__ void pull(const S* __restrict__ f, const uint16_t* __restrict__ flags,
                                     const Lat& lat, const Cell& c, long long n,
                                     typename St<S>::R fi[Q], unsigned& solid_links,
                                     uint16_t own_flag = F_NEAR) {
  const size_t N = (size_t)lat.Ns;  // population stride
  const bool near = (own_flag & F_NEAR) != 0;
  solid_links = 0;
  if constexpr (sizeof(S) == 2) {
    // binary16: all 19 raw loads are issued before any conversion (converting each value as it
    // arrives made every load wait for the one before: 2.5x slower); St<__half> adds the weight of
    // the direction actually read, and opp(i) has the same weight as i
    unsigned short raw[Q];
    raw[0] = __ldg(reinterpret_cast<const unsigned short*>(f) + n);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const long long s = nbr(c, lat, i, -1);
      const bool sol = near && (__ldg(flags + s) & F_SOLID);
      solid_links |= (unsigned)sol << i;
      raw[i] = __ldg(reinterpret_cast<const unsigned short*>(f) + (sol ? (size_t)opp_of(i) * N + n : (size_t)i * N + s));
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) fi[i] = St<S>::from_raw(raw[i], i);
  } else {
    fi[0] = St<S>::ld(f, (size_t)n, 0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const long long s = nbr(c, lat, i, -1);
      const bool sol = near && (__ldg(flags + s) & F_SOLID);
      solid_links |= (unsigned)sol << i;
      fi[i] = St<S>::ld(f, sol ? (size_t)opp_of(i) * N + n : (size_t)i * N + s, i);
    }
  }
}

// Guo-forced BGK collision (Eqs. lb_collision, distribution_eq, guo_forcing) of one cell, written
// to dst. Opposite directions share the even part of f_eq + F_i and flip the odd part:
// f*_i = (1 - 1/tau) f_i + S_i + A_i, f*_opp = (1 - 1/tau) f_opp + S_i - A_i with
// S_i = (rho w_i / tau)(1 + 4.5 (c.v)^2 - 1.5 v.v) + (1 - 1/2tau) w_i (9 (c.v)(c.F) - 3 v.F),
// A_i = 3 w_i ((rho / tau) c.v + (1 - 1/2tau) c.F).
// Post-collision values of one cell, handed to sink(i, v) in direction order.
// Weight w_i in the arithmetic type of a kernel: the FP32 set whose values sum to exactly 1 (so the
// equilibria of an FP32 collision add no mass, weights.h), or the FP64 value.
template <typename R>
__device__ __forceinline__ R wgt(int i) {
  if constexpr (sizeof(R) == 8) {
    return (R)w_of(i);
  } else {
    return wf_of(i);
  }
}

template <typename R, typename Sink>
__device__ __forceinline__ void bgk_values(const R fi[Q], R rho, R vx, R vy, R vz, R Fx, R Fy, R Fz, R tau,
                                           const Sink& sink) {
  const R itau = (R)1 / tau;
  const R keep = (R)1 - itau;
  const R pref = (R)1 - (R)0.5 * itau;
  const R ro = rho * itau;
  const R uu = vx * vx + vy * vy + vz * vz;
  const R vF = vx * Fx + vy * Fy + vz * Fz;
  const R base = (R)1 - (R)1.5 * uu;   // even part without (c.v)^2
  const R fv = -(R)3 * pref * vF;       // even forcing part without (c.v)(c.F)
  sink(0, keep * fi[0] + wgt<R>(0) * (ro * base + fv));
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const R cu = (R)cx_of(i) * vx + (R)cy_of(i) * vy + (R)cz_of(i) * vz;
    const R cF = (R)cx_of(i) * Fx + (R)cy_of(i) * Fy + (R)cz_of(i) * Fz;
    const R w = wgt<R>(i);
    const R sym = w * (ro * (base + (R)4.5 * cu * cu) + fv + (R)9 * pref * cu * cF);
    const R anti = (R)3 * w * (ro * cu + pref * cF);
    sink(i, keep * fi[i] + sym + anti);
    sink(i + 1, keep * fi[i + 1] + sym - anti);
  }
}

// OUT: fo receives the stored values as a later load returns them (the accumulating pass sums them
// into the next step's density).
template <typename S, bool OUT = false>
__device__ __forceinline__ void collide_store(S* __restrict__ dst, size_t N, long long n,
                                              const typename St<S>::R fi[Q], typename St<S>::R rho,
                                              typename St<S>::R vx, typename St<S>::R vy, typename St<S>::R vz,
                                              typename St<S>::R Fx, typename St<S>::R Fy, typename St<S>::R Fz,
                                              typename St<S>::R tau, typename St<S>::R* fo = nullptr) {
  using R = typename St<S>::R;
  bgk_values<R>(fi, rho, vx, vy, vz, Fx, Fy, Fz, tau, [&](int i, R v) {
    St<S>::st(dst, (size_t)i * N + (size_t)n, i, v);
    if constexpr (OUT) fo[i] = St<S>::rt(v, i);
  });
}

template <typename S>
__global__ void __launch_bounds__(128) k_density(const S* __restrict__ fa, const S* __restrict__ fb,
                                                 const StepState* __restrict__ st,
                                                 const uint16_t* __restrict__ flags,
                                                 const BodyDev* __restrict__ bodies,
                                                 typename St<S>::R* __restrict__ psi_a,
                                                 typename St<S>::R* __restrict__ psi_b, Lat lat, double rho0,
                                                 float rho0_f) {
  using R = typename St<S>::R;
  const S* __restrict__ f = st->parity ? fb : fa;
  // two psi buffers (accumulating pass): the current step's is the one the parity names
  R* __restrict__ psi = (psi_b && st->parity) ? psi_b : psi_a;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
  if (x >= lat.nx || y >= lat.ny) return;
  const Cell c = make_cell(x, y, z, lat);
  const long long n = c.n;
  const uint16_t fl = flags[n];
  R ps;
  if (fl & F_SOLID) {
    ps = par<R>(bodies[fl & F_OWNER].psi_wet, bodies[fl & F_OWNER].psi_wet_f);
  } else {
    R fi[Q];
    unsigned sl;
    pull<S>(f, flags, lat, c, n, fi, sl, fl);
    R rho = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) rho += fi[i];
    ps = (R)1 - exp(-rho / par<R>(rho0, rho0_f));
  }
  psi[n] = ps;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of one value per lane, returned in FP64 to every lane. FP64 values go through the FP64
// butterfly. FP32 values go through an FP32 butterfly that carries each rounding error (Knuth's
// TwoSum, exact in round-to-nearest) in a second float, so the result is the exact warp sum to
// about 2^-48 relative without the 5 FP64 adds and the conversion per lane of the plain form
// (GB300 issues FP64 at 1/64 of the FP32 rate).
__device__ __forceinline__ double warp_mass(double v) { return warp_sum(v); }
__device__ __forceinline__ double warp_mass(float v) {
  float hi = v, lo = 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
    const float s = __fadd_rn(hi, bh);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, bl), err);
  }
  // every lane holds the same pair; only lane 0's result is used, so only lane 0 converts
  const unsigned lin = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  return (lin & 31) == 0 ? (double)hi + (double)lo : 0.0;
}

// minimum image of a coordinate difference in (-1.5 n, 1.5 n): one wrap gives the same result as
// repeated wrapping
template <typename R>
__device__ __forceinline__ R mimg1(R d, int n) {
  const R h = (R)0.5 * (R)n;
  if (d >= h) d -= (R)n;
  else if (d < -h) d += (R)n;
  return d;
}

// moving-wall term of solid link i at fluid cell c: g_i = 2 rho w_i c_i.u_B(x - c_i/2) / c_s^2
template <typename R>
__device__ __forceinline__ R wall_term(const BodyDev& b, const Cell& c, const Lat& lat, int i, R rho) {
  const R mx = (R)c.x - (R)0.5 * (R)cx_of(i), my = (R)c.y - (R)0.5 * (R)cy_of(i), mz = (R)c.z - (R)0.5 * (R)cz_of(i);
  const R ax = mimg1<R>(mx - par<R>(b.X[0], b.Xf[0]), lat.nx), ay = mimg1<R>(my - par<R>(b.X[1], b.Xf[1]), lat.ny),
          az = mimg1<R>(mz - par<R>(b.X[2], b.Xf[2]), lat.nz);
  const R wx = par<R>(b.W[0], b.Wf[0]), wy = par<R>(b.W[1], b.Wf[1]), wz = par<R>(b.W[2], b.Wf[2]);
  const R ux = par<R>(b.V[0], b.Vf[0]) + (wy * az - wz * ay);
  const R uy = par<R>(b.V[1], b.Vf[1]) + (wz * ax - wx * az);
  const R uz = par<R>(b.V[2], b.Vf[2]) + (wx * ay - wy * ax);
  const R cu = (R)cx_of(i) * ux + (R)cy_of(i) * uy + (R)cz_of(i) * uz;
  return (R)2 * rho * (R)w_of(i) * cu * (R)3;
}

// Resident 128-thread blocks per SM requested for the bulk collision kernel: for FP32 occupancy
// matters more than the few registers it spills (64 registers, a 20-byte spill; 7 blocks without a
// spill measure the same); FP64 needs more room.
#ifndef CBL_COLLIDE_MINB
#define CBL_COLLIDE_MINB 8
#endif
template <typename S>
struct CollideMinBlocks {
  static constexpr int value = CBL_COLLIDE_MINB;
};
template <>
struct CollideMinBlocks<double> {
  static constexpr int value = 4;
};
// binary16 storage: 7 blocks (72 registers) avoids a register spill that 8 blocks force, and is faster
template <>
struct CollideMinBlocks<__half> {
  static constexpr int value = 7;
};
// Collision of one fluid cell: Shan-Chen force with wetting, pull, moving-wall terms on solid links,
// Guo-forced BGK, store. NEAR: the cell has a solid neighbour along a lattice direction (bounce-back
// sources, wall terms, (rho, psi) for the force pass); without it the pull reads no flags at all, so
// the bulk kernel carries neither the flag loads (on which the population addresses would depend)
// nor the registers of the wall terms. Returns rho.
// psi_at(i): psi at x + c_i (i >= 1) and at x itself (i = 0).
// Shan-Chen force with wetting (Eq. shan_chen_force; solid neighbours carry psi of their wetting
// density) plus the external force. psi_at(i): psi at x + c_i (i >= 1) and at x (i = 0).
// The sum over directions is taken over opposite pairs (c_opp = -c_i, equal weights), as sums of
// differences psi(x + c_i) - psi(x - c_i): the same value, but its rounding scales with the small
// differences of psi across a cell, not with psi itself (in the bulk of a phase the terms cancel, and
// summing them one by one in FP32 would leave a rounding residue of ~1e-7 psi as a force).
template <typename R, typename PsiAt>
__device__ __forceinline__ void sc_force(const PsiAt& psi_at, const PhysParams& pp, R& ps, R& Fx, R& Fy, R& Fz) {
  ps = psi_at(0);
  R sx = 0, sy = 0, sz = 0;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const R wd = (R)w_of(i) * (psi_at(i) - psi_at(i + 1));
    if (cx_of(i)) sx += wd * (R)cx_of(i);
    if (cy_of(i)) sy += wd * (R)cy_of(i);
    if (cz_of(i)) sz += wd * (R)cz_of(i);
  }
  const R mG = -par<R>(pp.G, pp.G_f) * ps;
  Fx = mG * sx + par<R>(pp.ext[0], pp.ext_f[0]);
  Fy = mG * sy + par<R>(pp.ext[1], pp.ext_f[1]);
  Fz = mG * sz + par<R>(pp.ext[2], pp.ext_f[2]);
}

// Velocity with the half-force shift (Eq. fluid_velocity); the momentum, like the force, summed over
// opposite pairs as f_i - f_opp(i) (rounding of the order of the differences, not of the
// populations, which matters at the small velocities of these flows).
template <typename R>
__device__ __forceinline__ void fluid_velocity(const R fi[Q], R rho, R Fx, R Fy, R Fz, R& vx, R& vy, R& vz) {
  R mx = (R)0.5 * Fx, my = (R)0.5 * Fy, mz = (R)0.5 * Fz;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const R d = fi[i] - fi[i + 1];
    if (cx_of(i)) mx += (R)cx_of(i) * d;
    if (cy_of(i)) my += (R)cy_of(i) * d;
    if (cz_of(i)) mz += (R)cz_of(i) * d;
  }
  vx = vy = vz = (R)0;
  if (rho > (R)0) {
    const R ir = (R)1 / rho;
    vx = mx * ir;
    vy = my * ir;
    vz = mz * ir;
  }
}

template <typename S, bool NEAR, typename PsiAt, bool OUT = false>
__device__ __forceinline__ typename St<S>::R collide_fluid(const S* __restrict__ src, S* __restrict__ dst,
                                                           const uint16_t* __restrict__ flags,
                                                           const PsiAt& psi_at,
                                                           const BodyDev* __restrict__ bodies, int diag,
                                                           double* __restrict__ diag_rho,
                                                           double* __restrict__ diag_vel, const Lat& lat,
                                                           const PhysParams& pp,
                                                           RhoPsi<typename St<S>::R>* __restrict__ nbuf,
                                                           const Cell& c, long long n,
                                                           typename St<S>::R* fo = nullptr) {
  using R = typename St<S>::R;
  const size_t N = (size_t)lat.Ns;  // population stride
  R my_mass = 0;
  {
    // the force first: it needs only psi, so the populations are not yet live
    R ps, Fx, Fy, Fz;
    sc_force<R>(psi_at, pp, ps, Fx, Fy, Fz);
    R fi[Q];
    unsigned sl;
    pull<S>(src, flags, lat, c, n, fi, sl, NEAR ? F_NEAR : (uint16_t)0);
    R rho = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) rho += fi[i];
    my_mass = rho;
    if (sl) {
      if (NEAR) nbuf[n] = RhoPsi<R>{rho, ps};
      // moving-wall term on each solid link and the mass correction delta rho = -sum g_i on the
      // rest population (Eqs. lb_bounce_back_us, lb_bounce_back_mass)
      R drho = 0;
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        if (!(sl & (1u << i))) continue;
        const int B = __ldg(flags + nbr(c, lat, i, -1)) & F_OWNER;
        const R g = wall_term<R>(bodies[B], c, lat, i, rho);
        fi[i] += g;
        drho -= g;
      }
      fi[0] += drho;
    }
    R vx, vy, vz;
    fluid_velocity<R>(fi, rho, Fx, Fy, Fz, vx, vy, vz);
    collide_store<S, OUT>(dst, N, n, fi, rho, vx, vy, vz, Fx, Fy, Fz, par<R>(pp.tau, pp.tau_f), fo);
    if (diag) {
      diag_rho[n] = (double)rho;
      diag_vel[3 * n] = (double)vx;
      diag_vel[3 * n + 1] = (double)vy;
      diag_vel[3 * n + 2] = (double)vz;
    }
  }
  return my_mass;
}

// Block sum of the cells' densities, added into one of MASS_SLOTS slots (spreads the atomics); the
// body kernel adds the slots in a fixed order and clears them. FP64 values are summed in FP64; FP32
// values in compensated float pairs (exact to about 2^-48) up to one FP64 conversion per block
// (GB300 issues FP64 at 1/64 of the FP32 rate).
__device__ __forceinline__ void add_mass_slot(double* __restrict__ mass_part, double v, unsigned slot) {
  __shared__ double wsum[32];
  const int lin = threadIdx.x + blockDim.x * threadIdx.y;
  const double m = warp_sum(v);
  if ((lin & 31) == 0) wsum[lin >> 5] = m;
  __syncthreads();
  if (lin == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)((blockDim.x * blockDim.y) >> 5); ++w) t += wsum[w];
    if (t != 0.0) atomicAdd(mass_part + (slot & (MASS_SLOTS - 1)), t);
  }
}
// the same from a compensated pair (hi, lo) per thread
__device__ __forceinline__ void add_mass_slot2(double* __restrict__ mass_part, float hi, float lo, unsigned slot) {
  __shared__ float whi[32], wlo[32];
  const int lin = threadIdx.x + blockDim.x * threadIdx.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
    const float s = __fadd_rn(hi, bh);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, bl), err);
  }
  if ((lin & 31) == 0) {
    whi[lin >> 5] = hi;
    wlo[lin >> 5] = lo;
  }
  __syncthreads();
  if (lin == 0) {
    float h = 0.0f, l = 0.0f;
    for (int w = 0; w < (int)((blockDim.x * blockDim.y) >> 5); ++w) {
      const float s = __fadd_rn(h, whi[w]);
      const float bb = __fsub_rn(s, h);
      const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(whi[w], bb));
      h = s;
      l = __fadd_rn(__fadd_rn(l, wlo[w]), err);
    }
    const double t = (double)h + (double)l;
    if (t != 0.0) atomicAdd(mass_part + (slot & (MASS_SLOTS - 1)), t);
  }
}
__device__ __forceinline__ void add_mass_slot(double* __restrict__ mass_part, float v, unsigned slot) {
  add_mass_slot2(mass_part, v, 0.0f, slot);
}

// fluid-mass accumulation of one thread over several cells: FP64 as it is, FP32 in a compensated
// pair (Knuth's TwoSum per add), so a thread's partial sum keeps the precision of a single cell's
template <typename R>
struct MassAcc;
template <>
struct MassAcc<double> {
  double v = 0.0;
  __device__ void add(double x) { v += x; }
};
template <>
struct MassAcc<float> {
  float hi = 0.0f, lo = 0.0f;
  __device__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb)));
    hi = s;
  }
};

__device__ __forceinline__ void add_mass_slot(double* __restrict__ mass_part, const MassAcc<double>& a,
                                              unsigned slot) {
  add_mass_slot(mass_part, a.v, slot);
}
__device__ __forceinline__ void add_mass_slot(double* __restrict__ mass_part, const MassAcc<float>& a,
                                              unsigned slot) {
  add_mass_slot2(mass_part, a.hi, a.lo, slot);
}


// Bulk collision: solid cells store zeros, fluid cells without a solid neighbour collide; fluid cells
// next to a solid are left to k_collide_near.
template <typename S>
__global__ void __launch_bounds__(128, CollideMinBlocks<S>::value) k_collide(S* __restrict__ fa, S* __restrict__ fb,
                                                 const uint16_t* __restrict__ flags,
                                                 const typename St<S>::R* __restrict__ psi,
                                                 const BodyDev* __restrict__ bodies,
                                                 double* __restrict__ mass_part, const StepState* __restrict__ st,
                                                 double* __restrict__ diag_rho, double* __restrict__ diag_vel,
                                                 Lat lat, PhysParams pp,
                                                 RhoPsi<typename St<S>::R>* __restrict__ nbuf) {
  using R = typename St<S>::R;
  const size_t N = (size_t)lat.Ns;  // population stride
  const int diag = st->diag;
  const S* __restrict__ src = st->parity ? fb : fa;
  S* __restrict__ dst = st->parity ? fa : fb;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
  const bool valid = x < lat.nx && y < lat.ny;
  const Cell c = make_cell(valid ? x : 0, valid ? y : 0, z, lat);
  const long long n = c.n;
  R my_mass = 0;
  const uint16_t fl = valid ? flags[n] : (uint16_t)0;
  if (valid && (fl & F_SOLID)) {
#pragma unroll
    for (int i = 0; i < Q; ++i) St<S>::st(dst, (size_t)i * N + n, i, (R)0);
    if (diag) {
      diag_rho[n] = 0.0;
      diag_vel[3 * n] = 0.0;
      diag_vel[3 * n + 1] = 0.0;
      diag_vel[3 * n + 2] = 0.0;
    }
  } else if (valid && !(fl & F_NEAR)) {
    auto psi_at = [&](int i) -> R { return i ? psi[nbr(c, lat, i, +1)] : psi[n]; };
    my_mass = collide_fluid<S, false>(src, dst, flags, psi_at, bodies, diag, diag_rho, diag_vel, lat, pp, nbuf, c, n);
  }
  add_mass_slot(mass_part, my_mass, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z));
}

// Collision of the fluid cells next to a solid (the boundary-cell list built by the refill pass).
template <typename S>
__global__ void __launch_bounds__(128) k_collide_near(S* __restrict__ fa, S* __restrict__ fb,
                                                      const uint16_t* __restrict__ flags,
                                                      const typename St<S>::R* __restrict__ psi_a,
                                                      const typename St<S>::R* __restrict__ psi_b,
                                                      const BodyDev* __restrict__ bodies,
                                                      double* __restrict__ mass_part,
                                                      const StepState* __restrict__ st,
                                                      double* __restrict__ diag_rho, double* __restrict__ diag_vel,
                                                      const int* __restrict__ blist, Lat lat, PhysParams pp,
                                                      RhoPsi<typename St<S>::R>* __restrict__ nbuf) {
  using R = typename St<S>::R;
  const R* __restrict__ psi = (psi_b && st->parity) ? psi_b : psi_a;
  const int diag = st->diag;
  const S* __restrict__ src = st->parity ? fb : fa;
  S* __restrict__ dst = st->parity ? fa : fb;
  const unsigned count = st->nbnd;
  R my_mass = 0;
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    const long long n = blist[k];
    const Cell c = cell_of(n, lat);
    auto psi_at = [&](int i) -> R { return i ? psi[nbr(c, lat, i, +1)] : psi[n]; };
    my_mass += collide_fluid<S, true>(src, dst, flags, psi_at, bodies, diag, diag_rho, diag_vel, lat, pp, nbuf, c, n);
  }
  add_mass_slot(mass_part, my_mass, blockIdx.x * 7u + 3u);
}

// ---- accumulating pass (lbm_variant 2) ---------------------------------------------------------
// The force of step t needs psi of the post-streaming density at every neighbour (Sec. 3.2.3,
// Eq. mean_field_potential), so the split pass pulls every cell's populations twice per step: once
// for rho and psi, once for the collision. This pass computes the next step's density while it
// collides: rho_{t+1}(x) = sum_i f*_i(x - c_i) is the pull of the populations it stores.
//
// A block owns a region of 32 x TY columns and marches through sz planes along z. After colliding a
// plane it puts the stored post-collision values in shared memory; each thread then adds, for its
// own column, the values whose source lies in the region, into the targets one plane below, in and
// above (three running sums, one barrier per plane). A cell's sum is complete when all its sources
// lie in the region: the region's interior cells, whose psi_{t+1} = 1 - exp(-rho / rho0) this pass
// stores into the other psi buffer (read by no other block: a block's gather reaches one cell into
// its neighbours, which are edge cells there). The edge cells (first or last column, row or plane
// of the region) store the partial sum instead; the fix-up pass of the next step adds the sources
// outside the region. Cells whose sources include a cell next to a solid (collided on the side
// branch, not here) or a solid lie in a body's tile, and the tile pass of the next step recomputes
// their psi from the populations, as the split pass does.

// Sources of cell (x, y, z) that lie in its region: the test that splits the sum between this pass
// and the fix-up (no periodic wrap: a wrapped source counts as outside even in a one-region axis).
__device__ __forceinline__ bool acc_source_inside(int sx, int sy, int sz_, int x0, int y0, int zb, int nvx, int nvy,
                                                  int ze) {
  return sx >= x0 && sx < x0 + nvx && sy >= y0 && sy < y0 + nvy && sz_ >= zb && sz_ < ze;
}

template <typename S, int TY, int MINB>
__global__ void __launch_bounds__(32 * TY, MINB) k_collide_acc(S* __restrict__ fa, S* __restrict__ fb,
                                                                const uint16_t* __restrict__ flags,
                                                                typename St<S>::R* __restrict__ psi_a,
                                                                typename St<S>::R* __restrict__ psi_b,
                                                                typename St<S>::R* __restrict__ rhop,
                                                                const BodyDev* __restrict__ bodies,
                                                                double* __restrict__ mass_part,
                                                                const StepState* __restrict__ st,
                                                                double* __restrict__ diag_rho,
                                                                double* __restrict__ diag_vel, Lat lat,
                                                                PhysParams pp, int sz) {
  using R = typename St<S>::R;
  constexpr int NT = 32 * TY;
  extern __shared__ __align__(16) unsigned char acc_smem[];
  R* sf = reinterpret_cast<R*>(acc_smem);  // [2][Q - 1][NT]: stored values of the plane, by direction
  const size_t N = (size_t)lat.Ns;
  const int diag = st->diag;
  const int parity = st->parity;
  const S* __restrict__ src = parity ? fb : fa;
  S* __restrict__ dst = parity ? fa : fb;
  const R* __restrict__ psi = parity ? psi_b : psi_a;
  R* __restrict__ psi_next = parity ? psi_a : psi_b;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY, zb = blockIdx.z * sz;
  const int ze = min(zb + sz, lat.nz);
  const int nvx = min(32, lat.nx - x0), nvy = min(TY, lat.ny - y0);
  const bool valid = tx < nvx && ty < nvy;
  const int x = valid ? x0 + tx : x0, y = valid ? y0 + ty : y0;
  const bool edge = tx == 0 || tx == nvx - 1 || ty == 0 || ty == nvy - 1;
  const size_t col = (size_t)x + (size_t)lat.nx * (size_t)y, plane = (size_t)lat.nx * (size_t)lat.ny;
  R am = 0, a0 = 0, ap = 0;  // running sums of the targets one plane below, in and above
  MassAcc<R> mass;
  for (int z = zb; z < ze; ++z) {
    R fo[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fo[i] = (R)0;
    if (valid) {
      const Cell c = make_cell(x, y, z, lat);
      const long long n = c.n;
      const uint16_t fl = flags[n];
      if (fl & F_SOLID) {
#pragma unroll
        for (int i = 0; i < Q; ++i) St<S>::st(dst, (size_t)i * N + n, i, (R)0);
        if (diag) {
          diag_rho[n] = 0.0;
          diag_vel[3 * n] = 0.0;
          diag_vel[3 * n + 1] = 0.0;
          diag_vel[3 * n + 2] = 0.0;
        }
      } else if (!(fl & F_NEAR)) {
        auto psi_at = [&](int i) -> R { return i ? psi[nbr(c, lat, i, +1)] : psi[n]; };
        mass.add(collide_fluid<S, false, decltype(psi_at), true>(src, dst, flags, psi_at, bodies, diag, diag_rho,
                                                                 diag_vel, lat, pp, nullptr, c, n, fo));
      }
    }
    R* buf = sf + (size_t)(z & 1) * (Q - 1) * NT;
#pragma unroll
    for (int i = 1; i < Q; ++i) buf[(i - 1) * NT + threadIdx.x] = fo[i];
    // one barrier per plane: the buffers alternate, and a thread writes a buffer again only after
    // the next plane's barrier, which every reader of this plane has passed
    __syncthreads();
    a0 += fo[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int sx = tx - cx_of(i), sy = ty - cy_of(i);
      if (sx >= 0 && sx < nvx && sy >= 0 && sy < nvy) {
        const R v = buf[(i - 1) * NT + sy * 32 + sx];
        if (cz_of(i) > 0) ap += v;
        else if (cz_of(i) < 0) am += v;
        else a0 += v;
      }
    }
    if (z > zb && valid) {
      const size_t n = col + plane * (size_t)(z - 1);
      if (edge || z - 1 == zb) rhop[n] = am;
      else psi_next[n] = (R)1 - exp(-am / par<R>(pp.rho0, pp.rho0_f));
    }
    am = a0;
    a0 = ap;
    ap = (R)0;
  }
  if (valid) rhop[col + plane * (size_t)(ze - 1)] = am;  // the last plane: an edge plane
  add_mass_slot(mass_part, mass, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z));
}

// Fix-up of the accumulating pass, at the start of the next step: psi of the regions' edge cells
// from the partial sum and the populations of the sources outside the region (Eq. lb_streaming
// pulled from the stored buffer). The cells next to a solid and their neighbours are left to the
// tile pass that follows. One thread per edge cell, in three ranges: the regions' first and last
// planes (whole rows), the first and last rows of the other planes (whole rows), the first and last
// columns of the remaining rows.
struct AccGeom {
  int ty, sz, nxr, nyr, nzr;  // region extents in y and z; regions per axis
  long long n1, n2, n3;       // edge cells of the three ranges
};

inline AccGeom acc_geom(const Lat& lat, int ty, int sz) {
  AccGeom g;
  g.ty = ty;
  g.sz = sz;
  g.nxr = (lat.nx + 31) / 32;
  g.nyr = (lat.ny + ty - 1) / ty;
  g.nzr = (lat.nz + sz - 1) / sz;
  g.n1 = 2LL * g.nzr * lat.ny * lat.nx;
  g.n2 = 2LL * g.nyr * lat.nz * lat.nx;
  g.n3 = 2LL * g.nxr * lat.ny * lat.nz;
  return g;
}

template <typename S>
__global__ void __launch_bounds__(256) k_psi_fixup(const S* __restrict__ fa, const S* __restrict__ fb,
                                                   typename St<S>::R* __restrict__ psi_a,
                                                   typename St<S>::R* __restrict__ psi_b,
                                                   const typename St<S>::R* __restrict__ rhop,
                                                   const StepState* __restrict__ st, Lat lat, double rho0,
                                                   float rho0_f, AccGeom g) {
  using R = typename St<S>::R;
  if (st->psi_skip) return;
  const S* __restrict__ f = st->parity ? fb : fa;
  R* __restrict__ psi = st->parity ? psi_b : psi_a;
  const size_t N = (size_t)lat.Ns;
  const long long total = g.n1 + g.n2 + g.n3;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    if (k < g.n1) {
      // first (side 0) or last (side 1) plane of a region, whole plane
      const long long r = k / lat.nx;
      x = (int)(k - r * lat.nx);
      const long long q = r / lat.ny;
      y = (int)(r - q * lat.ny);
      const int zr = (int)(q >> 1), side = (int)(q & 1);
      const int zb = zr * g.sz, ze = min(zb + g.sz, lat.nz);
      if (side && ze - 1 == zb) continue;
      z = side ? ze - 1 : zb;
    } else if (k < g.n1 + g.n2) {
      // first or last row of a region, planes that are not a region's first or last
      const long long kk = k - g.n1;
      const long long r = kk / lat.nx;
      x = (int)(kk - r * lat.nx);
      const long long q = r / lat.nz;
      z = (int)(r - q * lat.nz);
      const int yr = (int)(q >> 1), side = (int)(q & 1);
      const int y0 = yr * g.ty, y1 = min(y0 + g.ty, lat.ny) - 1;
      if (side && y1 == y0) continue;
      y = side ? y1 : y0;
      const int zb = (z / g.sz) * g.sz, ze = min(zb + g.sz, lat.nz);
      if (z == zb || z == ze - 1) continue;
    } else {
      // first or last column of a region, rows and planes that are not a region's first or last
      const long long kk = k - g.n1 - g.n2;
      const int e = (int)(kk % (2 * g.nxr));
      const long long r = kk / (2 * g.nxr);
      y = (int)(r % lat.ny);
      z = (int)(r / lat.ny);
      const int x0 = (e >> 1) * 32, x1 = min(x0 + 32, lat.nx) - 1;
      if ((e & 1) && x1 == x0) continue;
      x = (e & 1) ? x1 : x0;
      const int zb = (z / g.sz) * g.sz, ze = min(zb + g.sz, lat.nz);
      if (z == zb || z == ze - 1) continue;
      const int y0 = (y / g.ty) * g.ty, y1 = min(y0 + g.ty, lat.ny) - 1;
      if (y == y0 || y == y1) continue;
    }
    const int x0 = x & ~31, y0 = (y / g.ty) * g.ty, zb = (z / g.sz) * g.sz;
    const int nvx = min(32, lat.nx - x0), nvy = min(g.ty, lat.ny - y0), ze = min(zb + g.sz, lat.nz);
    const Cell c = make_cell(x, y, z, lat);
    R rho = rhop[c.n];
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (!acc_source_inside(x - cx_of(i), y - cy_of(i), z - cz_of(i), x0, y0, zb, nvx, nvy, ze))
        rho += St<S>::ld(f, (size_t)i * N + (size_t)nbr(c, lat, i, -1), i);
    psi[c.n] = (R)1 - exp(-rho / par<R>(rho0, rho0_f));
  }
}

// the cell (gx, gy, gz) lies in the tile of a body with a lower id than `self` (so that a pass over
// the tiles visits every cell once)
__device__ __forceinline__ bool covered_by_lower(const BodyDev* bodies, const BodyDev& b, int self, int gx, int gy,
                                                 int gz, const Lat& lat) {
  for (int k = 0; k < b.nnb; ++k) {
    int o = b.nbl[k];
    if (o >= self) break;
    const BodyDev& ob = bodies[o];
    if (wrapi_near(gx - ob.o[0], lat.nx) < ob.L[0] && wrapi_near(gy - ob.o[1], lat.ny) < ob.L[1] &&
        wrapi_near(gz - ob.o[2], lat.nz) < ob.L[2])
      return true;
  }
  return false;
}

// ---- fused bulk pass: density, psi, Shan-Chen force and collision in one pass -----------------
// The Shan-Chen force at x needs psi of the post-streaming density of this step at all neighbours
// x + c_i (Eq. benzi_force), so every cell's populations are pulled twice per step: once for the
// density, once for the collision. The split path does that in two kernels, two passes over HBM.
// Here a block owns a TX x TY column of cells and marches along z over [z0, z0 + tz): for plane
// z + 1 it pulls the populations of its own cells and of the one-cell ring around them (periodic
// coordinates) and keeps only psi, in a ring of four planes in shared memory; then it collides plane
// z, pulling its own cells' populations again. That second pull comes one plane after the first and
// is served by the L1/L2 caches, and the ring cells are cells that neighbouring blocks own (L2), so
// HBM sees every population read once per step. Fluid cells next to a solid (F_NEAR) are left to
// k_collide_near, which reads psi from the lattice array that k_density_tiles fills over the bodies'
// tiles. The arithmetic is that of k_density + k_collide, term by term in the same order, so both
// paths give bit-identical results.

// psi of one cell from the current populations: the post-streaming density with half-way
// bounce-back at solid neighbours (Eq. lb_bounce_back; the g terms cancel in the density because of
// the mass correction), psi = 1 - exp(-rho / rho0) (Eq. mean_field_potential); a solid cell carries
// psi of its owner's wetting density (Sec. 3.2.3). The same expression as k_density.
template <typename S>
__device__ __forceinline__ typename St<S>::R psi_of_cell(const S* __restrict__ src, const uint16_t* __restrict__ flags,
                                                         const BodyDev* __restrict__ bodies, const Lat& lat,
                                                         const Cell& c, double rho0, float rho0_f) {
  using R = typename St<S>::R;
  const uint16_t fl = __ldg(flags + c.n);
  if (fl & F_SOLID) return par<R>(bodies[fl & F_OWNER].psi_wet, bodies[fl & F_OWNER].psi_wet_f);
  R fi[Q];
  unsigned sl;
  pull<S>(src, flags, lat, c, (long long)c.n, fi, sl, fl);
  R rho = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) rho += fi[i];
  return (R)1 - exp(-rho / par<R>(rho0, rho0_f));
}

// Named barriers of the fused pass's producer/consumer hand-off (barrier 0 is __syncthreads).
// bar.arrive marks the calling warp's arrival and does not wait; bar.sync waits for the barrier's
// generation to complete; once `count` threads have done either, the generation completes and the
// arriving threads' earlier shared-memory writes are visible to the waiting ones.
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Block layout: TX x TY consumer threads (warps 0 .. TY*TX/32 - 1), one per column of the tile,
// collide plane after plane; NPW producer warps behind them compute psi of the extended plane
// (tile + one-cell ring) up to K - 2 planes ahead, so the HBM latency of the producers' pulls
// overlaps the consumers' collisions. psi planes live in K shared-memory slots; FULL(s) hands slot
// s from the producers to the consumers, EMPTY(s) hands it back. Every barrier generation has all
// NALL threads: each producer thread arrives on FULL(slot of q) for every plane q and waits on
// EMPTY before overwriting a slot (planes q >= K); each consumer waits on FULL for every plane and
// releases plane j - 1 after colliding plane j (only while a producer will wait for it).
template <typename S, int TX, int TY, int NPW, int MINB>
__global__ void __launch_bounds__(TX * TY + 32 * NPW, MINB) k_fused(S* __restrict__ fa, S* __restrict__ fb,
                                                                     const uint16_t* __restrict__ flags,
                                                                     const BodyDev* __restrict__ bodies,
                                                                     double* __restrict__ mass_part,
                                                                     const StepState* __restrict__ st,
                                                                     double* __restrict__ diag_rho,
                                                                     double* __restrict__ diag_vel, Lat lat,
                                                                     PhysParams pp, int tz) {
  using R = typename St<S>::R;
  constexpr int NC = TX * TY, NP = 32 * NPW, NALL = NC + NP;
  constexpr int EX = TX + 2, EY = TY + 2, EP = EX * EY, MAXP = (EP + NP - 1) / NP;
  constexpr int K = 4;
  static_assert(NC % 32 == 0, "whole consumer warps");
  __shared__ R s_psi[K][EP];
  const int diag = st->diag;
  const S* __restrict__ src = st->parity ? fb : fa;
  S* __restrict__ dst = st->parity ? fa : fb;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * tz;
  const int zend = min(z0 + tz, lat.nz);
  const int J = zend - z0 + 1;  // planes z0 - 1 .. zend have indices 0 .. J
  MassAcc<R> mass;
  if (tid >= NC) {
    // producer: psi of extended cells p = ptid + k NP, for planes z0 - 1 .. zend
    const int ptid = tid - NC;
    int xs[MAXP], ys[MAXP];
#pragma unroll
    for (int k = 0; k < MAXP; ++k) {
      const int p = ptid + k * NP;
      xs[k] = wrapi(x0 - 1 + p % EX, lat.nx);
      ys[k] = wrapi(y0 - 1 + p / EX, lat.ny);
    }
    for (int j = 0; j <= J; ++j) {
      const int sl = j % K;
      if (j >= K) named_sync(1 + K + sl, NALL);
      const int zz = wrapi(z0 - 1 + j, lat.nz);
#pragma unroll
      for (int k = 0; k < MAXP; ++k) {
        const int p = ptid + k * NP;
        if (p < EP)
          s_psi[sl][p] = psi_of_cell<S>(src, flags, bodies, lat, make_cell(xs[k], ys[k], zz, lat), pp.rho0, pp.rho0_f);
      }
      named_arrive(1 + sl, NALL);
    }
  } else {
    // consumer: the collision of this thread's column
    const int tx = tid % TX, ty = tid / TX;
    const bool valid = x0 + tx < lat.nx && y0 + ty < lat.ny;
    const int p_own = (ty + 1) * EX + tx + 1;
    const int xo = valid ? x0 + tx : 0, yo = valid ? y0 + ty : 0;
    named_sync(1 + 0, NALL);  // plane z0 - 1
    for (int z = z0; z < zend; ++z) {
      const int j = z - z0 + 1;
      if (j == 1) named_sync(1 + 1 % K, NALL);  // plane z0
      named_sync(1 + (j + 1) % K, NALL);        // plane z + 1
      if (valid) {
        const Cell c = make_cell(xo, yo, z, lat);
        const long long n = c.n;
        const uint16_t fl = flags[n];
        if (fl & F_SOLID) {
          const size_t N = (size_t)lat.Ns;
#pragma unroll
          for (int i = 0; i < Q; ++i) St<S>::st(dst, (size_t)i * N + n, i, (R)0);
          if (diag) {
            diag_rho[n] = 0.0;
            diag_vel[3 * n] = 0.0;
            diag_vel[3 * n + 1] = 0.0;
            diag_vel[3 * n + 2] = 0.0;
          }
        } else if (!(fl & F_NEAR)) {
          const int s0 = j % K, sm = (j - 1) % K, sp = (j + 1) % K;
          auto psi_at = [&](int i) -> R {
            if (i == 0) return s_psi[s0][p_own];
            const int sl = cz_of(i) > 0 ? sp : (cz_of(i) < 0 ? sm : s0);
            return s_psi[sl][p_own + cy_of(i) * EX + cx_of(i)];
          };
          mass.add(collide_fluid<S, false>(src, dst, flags, psi_at, bodies, diag, diag_rho, diag_vel, lat, pp,
                                           nullptr, c, n));
        }
      }
      // plane j - 1 is no longer read; hand it back if a producer will reuse its slot
      if (j - 1 <= J - K) named_arrive(1 + K + (j - 1) % K, NALL);
    }
  }
  add_mass_slot(mass_part, mass, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z));
}

// psi of every cell of the bodies' tiles (each cell once: the lowest-id tile that covers it), for
// the collision of the cells next to a solid on the side branch of the fused step
template <typename S>
__global__ void __launch_bounds__(256) k_density_tiles(const S* __restrict__ fa, const S* __restrict__ fb,
                                                       const StepState* __restrict__ st,
                                                       const uint16_t* __restrict__ flags,
                                                       const BodyDev* __restrict__ bodies,
                                                       typename St<S>::R* __restrict__ psi_a,
                                                       typename St<S>::R* __restrict__ psi_b, Lat lat,
                                                       double rho0, float rho0_f) {
  // accumulating pass: nothing to do in a step whose psi a whole-lattice density pass computed
  if (psi_b && st->psi_skip) return;
  const S* __restrict__ f = st->parity ? fb : fa;
  typename St<S>::R* __restrict__ psi = (psi_b && st->parity) ? psi_b : psi_a;
  const int self = blockIdx.y;
  const BodyDev& b = bodies[self];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b.sz) return;
  const unsigned u = (unsigned)t, L0 = (unsigned)b.L[0], L1 = (unsigned)b.L[1];  // tiles hold < 2^31 cells
  const unsigned r = u / L0;
  const int gx = wrapi_near(b.o[0] + (int)(u - r * L0), lat.nx), gy = wrapi_near(b.o[1] + (int)(r % L1), lat.ny),
            gz = wrapi_near(b.o[2] + (int)(r / L1), lat.nz);
  if (b.nnb && covered_by_lower(bodies, b, self, gx, gy, gz, lat)) return;
  const Cell c = make_cell(gx, gy, gz, lat);
  psi[c.n] = psi_of_cell<S>(f, flags, bodies, lat, c, rho0, rho0_f);
}

// compensated float sum (Knuth's TwoSum): hi + lo carries the exact sum of the added values to about
// 2^-48 relative, so the per-body sums keep FP64-level accuracy while only the last step per block
// runs on the FP64 pipe (GB300 issues FP64 at 1/64 of the FP32 rate)
struct Sum2 {
  float hi, lo;
};
__device__ __forceinline__ Sum2 sum2_add(Sum2 a, Sum2 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return Sum2{s, __fadd_rn(__fadd_rn(a.lo, b.lo), err)};
}
template <typename R>
struct LinkSum;
template <>
struct LinkSum<float> {
  Sum2 v;
  __device__ void set(float x) { v = Sum2{x, 0.0f}; }
  __device__ void add(const LinkSum& o) { v = sum2_add(v, o.v); }
  __device__ LinkSum shfl_xor(int m) const {
    LinkSum r;
    r.v.hi = __shfl_xor_sync(0xffffffffu, v.hi, m);
    r.v.lo = __shfl_xor_sync(0xffffffffu, v.lo, m);
    return r;
  }
  __device__ double value() const { return (double)v.hi + (double)v.lo; }
};
template <>
struct LinkSum<double> {
  double v;
  __device__ void set(double x) { v = x; }
  __device__ void add(const LinkSum& o) { v += o.v; }
  __device__ LinkSum shfl_xor(int m) const {
    LinkSum r;
    r.v = __shfl_xor_sync(0xffffffffu, v, m);
    return r;
  }
  __device__ double value() const { return v; }
};

// ---- persistent lattice-Boltzmann pass over a batch of lattices ---------------------------------
// One launch for every instance of a batch: the grid is as large as the GPU holds at once (every
// block resident), and each block takes work items (one tile of TX x TY x TZ cells of one instance)
// from a device queue until none are left. Phase 0 computes psi of every cell of every instance (as
// k_density); a grid barrier follows, since a cell's force needs psi of cells that other blocks
// computed; phase 1 collides every cell without a solid neighbour (as k_collide). The barrier's wait
// is bounded: a block that has waited spin_limit cycles sets err bit 0 and returns, and so does every
// block once err is set, so an incomplete barrier ends the launch instead of hanging it.
__device__ __forceinline__ bool grid_barrier(BatchCtl* ctl) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = &ctl->gen;
    const unsigned gen = *vgen;  // read before arriving: the last arrival needs this block's
    __threadfence();
    if (atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1) {
      atomicExch(&ctl->arrive, 0u);
      __threadfence();
      atomicAdd(&ctl->gen, 1u);
    } else {
      const long long t0 = clock64(), limit = ctl->spin_limit;
      while (*vgen == gen) {
        if (clock64() - t0 > limit) {
          atomicOr(&ctl->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(256);
      }
    }
    __threadfence();
    if (*(volatile int*)&ctl->err) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename S, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX * TY, CollideMinBlocks<S>::value)
    k_batch_lbm(const BatchInst* __restrict__ tab, int ninst, long long items, BatchCtl* ctl) {
  using R = typename St<S>::R;
  __shared__ long long s_item;
  for (int phase = 0; phase < 2; ++phase) {
    if (phase == 1 && !grid_barrier(ctl)) return;
    for (;;) {
      if (threadIdx.x == 0) s_item = (long long)atomicAdd(&ctl->queue[phase], 1ull);
      __syncthreads();
      const long long item = s_item;
      __syncthreads();  // s_item is written again in the next round
      if (item >= items) break;
      // the instance whose items contain this one (item0 ascends with the instance index)
      int lo = 0, hi = ninst - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].item0 <= item) lo = mid;
        else hi = mid - 1;
      }
      const BatchInst& I = tab[lo];
      const Lat lat = I.lat;
      const long long k = item - I.item0;
      const int bx = (int)(k % I.tiles[0]), by = (int)((k / I.tiles[0]) % I.tiles[1]),
                bz = (int)(k / ((long long)I.tiles[0] * I.tiles[1]));
      const int x = bx * TX + (int)(threadIdx.x % TX), y = by * TY + (int)(threadIdx.x / TX);
      const bool valid = x < lat.nx && y < lat.ny;
      const StepState* st = I.st;
      const S* __restrict__ src = (const S*)(st->parity ? I.fb : I.fa);
      R* __restrict__ psi = (R*)I.psi;
      const int z0 = bz * TZ, z1 = min(z0 + TZ, lat.nz);
      if (phase == 0) {
        if (valid)
          for (int z = z0; z < z1; ++z) {
            const Cell c = make_cell(x, y, z, lat);
            psi[c.n] = psi_of_cell<S>(src, I.flags, I.bodies, lat, c, I.pp.rho0, I.pp.rho0_f);
          }
      } else {
        S* __restrict__ dst = (S*)(st->parity ? I.fa : I.fb);
        const int diag = st->diag;
        const size_t N = (size_t)lat.Ns;
        MassAcc<R> mass;
        if (valid)
          for (int z = z0; z < z1; ++z) {
            const Cell c = make_cell(x, y, z, lat);
            const long long n = c.n;
            const uint16_t fl = I.flags[n];
            if (fl & F_SOLID) {
#pragma unroll
              for (int i = 0; i < Q; ++i) St<S>::st(dst, (size_t)i * N + n, i, (R)0);
              if (diag) {
                I.diag_rho[n] = 0.0;
                I.diag_vel[3 * n] = 0.0;
                I.diag_vel[3 * n + 1] = 0.0;
                I.diag_vel[3 * n + 2] = 0.0;
              }
            } else if (!(fl & F_NEAR)) {
              auto psi_at = [&](int i) -> R { return i ? psi[nbr(c, lat, i, +1)] : psi[n]; };
              mass.add(collide_fluid<S, false>(src, dst, I.flags, psi_at, I.bodies, diag, I.diag_rho, I.diag_vel, lat,
                                               I.pp, nullptr, c, n));
            }
          }
        add_mass_slot(I.mass_part, mass, (unsigned)k);
      }
    }
  }
}

// ---- solid-fluid force on the bodies ---------------------------------------------------------
// For each listed fluid cell x: for a solid upstream neighbour s = x - c_i (owner B), momentum
// exchange -c_i (2 f*_opp(i)(x) + g_i) with the arm at the link midpoint (Eq. solid_liquid_force);
// for a solid downstream neighbour x + c_i (owner B), the reaction of the Shan-Chen force,
// +G psi(x) w_i psi(x + c_i) c_i, arm x + c_i - X_B (Sec. 3.2.3). It reads the same source
// populations and psi as the collision, so g_i and rho are bit-identical to the ones it used.
// One thread per (list cell, direction): ~18x the parallelism of a thread per cell, which matters
// because the list is short (the fluid cells next to a solid) and each link's work is a chain of
// dependent loads (flags -> population or body). The 12 sums per body (momentum exchange F, T;
// adhesion F, T) are reduced in compensated precision over the warp and the block and added to the
// FP64 accumulators once per block and body.
template <typename S>
__global__ void __launch_bounds__(256) k_boundary(const S* __restrict__ fa, const S* __restrict__ fb,
                                                  const uint16_t* __restrict__ flags,
                                                  const BodyDev* __restrict__ bodies, double* __restrict__ acc,
                                                  const int* __restrict__ blist, const StepState* __restrict__ st,
                                                  const RhoPsi<typename St<S>::R>* __restrict__ nbuf, Lat lat,
                                                  double G, float G_f) {
  using R = typename St<S>::R;
  constexpr int NW = 8;  // warps per block
  __shared__ LinkSum<R> part[NW][12];
  __shared__ int pown[NW];
  const unsigned total = st->nbnd * (unsigned)(Q - 1);
  const S* __restrict__ src = st->parity ? fb : fa;
  const size_t N = (size_t)lat.Ns;  // population stride
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // whole-block rounds so that every thread reaches the barriers
  for (unsigned base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
    const unsigned k = base + threadIdx.x;
    R v[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) v[q] = 0;
    int Bm = -1, Ba = -1;  // body of the momentum-exchange term, of the adhesion term
    if (k < total) {
      const unsigned cell = k / (unsigned)(Q - 1);
      const int i = 1 + (int)(k - cell * (unsigned)(Q - 1));
      const long long n = blist[cell];
      const Cell c = cell_of(n, lat);
      const uint16_t up = __ldg(flags + nbr(c, lat, i, -1)), dn = __ldg(flags + nbr(c, lat, i, +1));
      if (up & F_SOLID) {
        // link to a solid upstream: the pulled value is f*_opp(i)(x) (half-way bounce-back)
        const int B = up & F_OWNER;
        const BodyDev& b = bodies[B];
        const RhoPsi<R> rp = nbuf[n];
        const R fi = St<S>::ld(src, (size_t)opp_of(i) * N + n, i);
        const R g = wall_term<R>(b, c, lat, i, rp.rho);
        const R m2 = (R)2 * fi + g;
        const R dPx = -(R)cx_of(i) * m2, dPy = -(R)cy_of(i) * m2, dPz = -(R)cz_of(i) * m2;
        const R ax = mimg1<R>((R)c.x - (R)0.5 * (R)cx_of(i) - par<R>(b.X[0], b.Xf[0]), lat.nx);
        const R ay = mimg1<R>((R)c.y - (R)0.5 * (R)cy_of(i) - par<R>(b.X[1], b.Xf[1]), lat.ny);
        const R az = mimg1<R>((R)c.z - (R)0.5 * (R)cz_of(i) - par<R>(b.X[2], b.Xf[2]), lat.nz);
        v[0] = dPx;
        v[1] = dPy;
        v[2] = dPz;
        v[3] = ay * dPz - az * dPy;
        v[4] = az * dPx - ax * dPz;
        v[5] = ax * dPy - ay * dPx;
        Bm = B;
      }
      if (dn & F_SOLID) {
        // solid downstream: reaction of the Shan-Chen force on that body
        const int B = dn & F_OWNER;
        const BodyDev& b = bodies[B];
        const R ps = nbuf[n].psi;
        const R gpw = par<R>(G, G_f) * ps * ((R)w_of(i) * par<R>(b.psi_wet, b.psi_wet_f));
        const R fx = gpw * (R)cx_of(i), fy = gpw * (R)cy_of(i), fz = gpw * (R)cz_of(i);
        const R ax = mimg1<R>((R)c.x + (R)cx_of(i) - par<R>(b.X[0], b.Xf[0]), lat.nx);
        const R ay = mimg1<R>((R)c.y + (R)cy_of(i) - par<R>(b.X[1], b.Xf[1]), lat.ny);
        const R az = mimg1<R>((R)c.z + (R)cz_of(i) - par<R>(b.X[2], b.Xf[2]), lat.nz);
        v[6] = fx;
        v[7] = fy;
        v[8] = fz;
        v[9] = ay * fz - az * fy;
        v[10] = az * fx - ax * fz;
        v[11] = ax * fy - ay * fx;
        Ba = B;
      }
    }
    // one body for the whole warp (the usual case): compensated warp sums; otherwise per-lane
    // FP64 atomics
    const int Bt = Bm >= 0 ? Bm : Ba;
    const bool mixed = Bm >= 0 && Ba >= 0 && Bm != Ba;
    const unsigned any = __ballot_sync(0xffffffffu, Bt >= 0);
    int b0 = -1;
    if (any) {
      b0 = __shfl_sync(0xffffffffu, Bt, __ffs(any) - 1);
      if (!__all_sync(0xffffffffu, (Bt < 0 || Bt == b0) && !mixed)) {
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          const int B = q < 6 ? Bm : Ba;
          if (B >= 0 && v[q] != (R)0) atomicAdd(acc + (size_t)B * ACC_N + q, (double)v[q]);
        }
        b0 = -1;
      } else {
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          LinkSum<R> a;
          a.set(v[q]);
#pragma unroll
          for (int m = 16; m > 0; m >>= 1) a.add(a.shfl_xor(m));
          if (lane == 0) part[w][q] = a;
        }
      }
    }
    if (lane == 0) pown[w] = b0;
    __syncthreads();
    if (threadIdx.x < 12) {
      // warps of the same body in a row are combined before one FP64 atomic
      const int q = threadIdx.x;
      int cur = -1;
      LinkSum<R> run;
      run.set((R)0);
      for (int ww = 0; ww < NW; ++ww) {
        const int B = pown[ww];
        if (B < 0) continue;
        if (B != cur) {
          if (cur >= 0) {
            const double x = run.value();
            if (x != 0.0) atomicAdd(acc + (size_t)cur * ACC_N + q, x);
          }
          cur = B;
          run.set((R)0);
        }
        run.add(part[ww][q]);
      }
      if (cur >= 0) {
        const double x = run.value();
        if (x != 0.0) atomicAdd(acc + (size_t)cur * ACC_N + q, x);
      }
    }
    __syncthreads();
  }
}

template <typename S>
__global__ void k_init_fluid(S* __restrict__ f, const uint16_t* __restrict__ flags, const double* __restrict__ rho,
                             const double* __restrict__ u, Lat lat) {
  using R = typename St<S>::R;
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= lat.N) return;
  const size_t N = (size_t)lat.Ns;  // population stride
  if (flags[n] & F_SOLID) {
#pragma unroll
    for (int i = 0; i < Q; ++i) St<S>::st(f, (size_t)i * N + n, i, (R)0);
    return;
  }
  double r = rho[n];
  if (!u) {
    // at rest: f_eq = rho w_i exactly (the bracket below is exactly 1), without its FP64 arithmetic
#pragma unroll
    for (int i = 0; i < Q; ++i) St<S>::st(f, (size_t)i * N + n, i, (R)(r * w_of(i)));
    return;
  }
  double ux = u[3 * n], uy = u[3 * n + 1], uz = u[3 * n + 2];
  double uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    double cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
    St<S>::st(f, (size_t)i * N + n, i, (R)(r * w_of(i) * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)));
  }
}


// ---- cover refill and boundary list ------------------------------------------------------------
// Over the body tiles (each cell once: the lowest-id tile that covers it), after the new flags.
// A fluid cell with a solid neighbour along a lattice direction goes into the boundary list of the
// next step. If any node was covered in this step, a fluid cell next to a covered node n receives
// f_eq(rho_n, u_n) / |N_F(n)| (face neighbours; all 26 if n has no fluid face neighbour).
template <typename S>
__global__ void __launch_bounds__(256) k_refill(S* __restrict__ fa, S* __restrict__ fb,
                                                uint16_t* __restrict__ flags,
                                                const BodyDev* __restrict__ bodies, StepState* st, int* blist,
                                                Lat lat, const double* __restrict__ arena, double member_thr,
                                                int* __restrict__ mbox, int next) {
  using R = typename St<S>::R;
  // the current state: the buffer this step's collision wrote (next = 1: the parity flips at the end
  // of the step) or, outside a step, the buffer the parity names
  S* __restrict__ f = (st->parity ^ next) ? fb : fa;
  const int self = blockIdx.y;
  const BodyDev& b = bodies[self];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  bool boundary = false;
  long long m = 0;
  // member cells (phi >= member_thr) of this body: their tile-coordinate bounding box, for the
  // repulsion pass of the next step
  bool member = false;
  int mi[3] = {0, 0, 0};
  float r2 = 0.0f;  // squared distance of a member cell from the body's centre
  if (t < b.sz) {
    const unsigned u = (unsigned)t, L0 = (unsigned)b.L[0], L1 = (unsigned)b.L[1];  // tiles hold < 2^31 cells
    const unsigned r = u / L0;
    const int i0 = (int)(u - r * L0), i1 = (int)(r % L1), i2 = (int)(r / L1);
    member = dbits(arena[b.off + t]) >= dbits(member_thr);
    mi[0] = i0;
    mi[1] = i1;
    mi[2] = i2;
    const int gx = wrapi_near(b.o[0] + i0, lat.nx), gy = wrapi_near(b.o[1] + i1, lat.ny),
              gz = wrapi_near(b.o[2] + i2, lat.nz);
    m = gx + (long long)lat.nx * (gy + (long long)lat.ny * gz);
    if (member) {
      // in float from the float mirror of X (FP64 is 1/64 rate here and this is a bound with slack);
      // tile cells lie within half a lattice length of X along each axis, so one wrap suffices
      const float dx = mimg1<float>((float)gx - b.Xf[0], lat.nx), dy = mimg1<float>((float)gy - b.Xf[1], lat.ny),
                  dz = mimg1<float>((float)gz - b.Xf[2], lat.nz);
      r2 = dx * dx + dy * dy + dz * dz;
    }
    if (!(b.nnb && covered_by_lower(bodies, b, self, gx, gy, gz, lat))) {
      const Cell c = cell_of(m, lat);
      const uint16_t fm = flags[m];
      const bool events = st->ncover != 0;
      const size_t N = (size_t)lat.Ns;  // population stride
      auto at = [&](int x, int y, int z) {
        return (long long)wrapi_near(x, lat.nx) +
               (long long)lat.nx * (wrapi_near(y, lat.ny) + (long long)lat.ny * wrapi_near(z, lat.nz));
      };
      auto fluid_count = [&](int x, int y, int z, bool faces_only) {
        int cnt = 0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int d2 = dx * dx + dy * dy + dz * dz;
              if (d2 == 0 || (faces_only && d2 > 1)) continue;
              if (!(flags[at(x + dx, y + dy, z + dz)] & F_SOLID)) cnt++;
            }
        return cnt;
      };
      if (fm & F_SOLID) {
        // a covered node with no fluid node within sqrt(3) loses its mass: count it
        if ((fm & F_COVER) && fluid_count(gx, gy, gz, false) == 0) {
          atomicAdd(&st->lost_refills, 1ull);
          atomicOr(&st->err, E_REFILL);
        }
      } else {
#pragma unroll
        for (int i = 1; i < Q; ++i) boundary |= (__ldg(flags + nbr(c, lat, i, +1)) & F_SOLID) != 0;
        // this thread is the only writer of the cell's flag word in this pass; concurrent readers
        // only test the solid bit, which this store does not change
        if (boundary != ((fm & F_NEAR) != 0)) flags[m] = boundary ? (uint16_t)(fm | F_NEAR) : (uint16_t)(fm & ~F_NEAR);
        if (events) {
          bool any = false;
          for (int dz = -1; dz <= 1 && !any; ++dz)
            for (int dy = -1; dy <= 1 && !any; ++dy)
              for (int dx = -1; dx <= 1 && !any; ++dx)
                if ((dx | dy | dz) && (flags[c.n + (unsigned)(c.ox[dx + 1] + c.oy[dy + 1] + c.oz[dz + 1])] & F_COVER))
                  any = true;
          if (any) {
            R add[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) add[i] = 0;
            for (int dz = -1; dz <= 1; ++dz)
              for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                  const int d2 = dx * dx + dy * dy + dz * dz;
                  if (d2 == 0) continue;
                  const int nxp = gx + dx, nyp = gy + dy, nzp = gz + dz;
                  const long long nn = c.n + (unsigned)(c.ox[dx + 1] + c.oy[dy + 1] + c.oz[dz + 1]);
                  if (!(flags[nn] & F_COVER)) continue;
                  const int c6 = fluid_count(nxp, nyp, nzp, true);
                  int cnt;
                  if (c6 > 0) {
                    if (d2 != 1) continue;  // only face neighbours share this node's populations
                    cnt = c6;
                  } else {
                    cnt = fluid_count(nxp, nyp, nzp, false);
                  }
                  R fi[Q];
                  R rho = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
                  for (int i = 0; i < Q; ++i) {
                    fi[i] = St<S>::ld(f, (size_t)i * N + nn, i);
                    rho += fi[i];
                    mx += (R)cx_of(i) * fi[i];
                    my += (R)cy_of(i) * fi[i];
                    mz += (R)cz_of(i) * fi[i];
                  }
                  R ux = 0, uy = 0, uz = 0;
                  if (rho > (R)0) {
                    ux = mx / rho;
                    uy = my / rho;
                    uz = mz / rho;
                  }
                  const R uu = ux * ux + uy * uy + uz * uz;
                  const R inv = (R)1 / (R)cnt;
#pragma unroll
                  for (int i = 0; i < Q; ++i) {
                    const R cu = (R)cx_of(i) * ux + (R)cy_of(i) * uy + (R)cz_of(i) * uz;
                    add[i] += rho * wgt<R>(i) * ((R)1 + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * uu) * inv;
                  }
                }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
              const size_t k = (size_t)i * N + m;
              St<S>::st(f, k, i, St<S>::ld(f, k, i) + add[i]);
            }
          }
        }
      }
    }
  }
  // warp, then block, then one set of global atomics per block (all warps of a block hit the same
  // six words, so per-warp global atomics would queue up)
  __shared__ int sbox[7];
  if (threadIdx.x < 7) sbox[threadIdx.x] = threadIdx.x < 3 ? INT_MAX : (threadIdx.x < 6 ? INT_MIN : 0);
  __syncthreads();
  if (__ballot_sync(0xffffffffu, member)) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int lo = __reduce_min_sync(0xffffffffu, member ? mi[a] : INT_MAX);
      const int hi = __reduce_max_sync(0xffffffffu, member ? mi[a] : INT_MIN);
      if (lane == 0) {
        atomicMin(sbox + a, lo);
        atomicMax(sbox + 3 + a, hi);
      }
    }
    // non-negative floats order like their bit patterns
    const unsigned rb = __reduce_max_sync(0xffffffffu, member ? __float_as_uint(r2) : 0u);
    if (lane == 0) atomicMax(sbox + 6, (int)rb);
  }
  __syncthreads();
  if (threadIdx.x < 7 && sbox[0] <= sbox[3]) {
    if (threadIdx.x < 3) atomicMin(mbox + MBOX_N * self + threadIdx.x, sbox[threadIdx.x]);
    else atomicMax(mbox + MBOX_N * self + threadIdx.x, sbox[threadIdx.x]);
  }
  // warp-aggregated append to the boundary list
  const unsigned mask = __ballot_sync(0xffffffffu, boundary);
  if (mask) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(&st->nbnd, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (boundary) blist[base + __popc(mask & ((1u << lane) - 1))] = (int)m;
  }
}

// current populations, widened to double, [direction][cell]; solid cells read zero (a node covered
// in the last step keeps its stale populations until the next collision overwrites them)
template <typename S>
__global__ void k_read_pop(const S* __restrict__ fa, const S* __restrict__ fb, const StepState* __restrict__ st,
                           const uint16_t* __restrict__ flags, double* __restrict__ out, Lat lat) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= lat.N) return;
  const S* f = st->parity ? fb : fa;
  const bool solid = flags[n] & F_SOLID;
#pragma unroll
  for (int i = 0; i < Q; ++i)
    out[(size_t)i * lat.N + n] = solid ? 0.0 : (double)St<S>::ld(f, (size_t)i * lat.Ns + n, i);
}

void launch_read_populations(int prec, const Lat& lat, const void* fa, const void* fb, const StepState* st,
                             const uint16_t* flags, double* out, cudaStream_t s) {
  const unsigned blocks = (unsigned)((lat.N + 255) / 256);
  if (prec == 0)
    k_read_pop<double><<<blocks, 256, 0, s>>>((const double*)fa, (const double*)fb, st, flags, out, lat);
  else if (prec == 1)
    k_read_pop<float><<<blocks, 256, 0, s>>>((const float*)fa, (const float*)fb, st, flags, out, lat);
  else
    k_read_pop<__half><<<blocks, 256, 0, s>>>((const __half*)fa, (const __half*)fb, st, flags, out, lat);
}

// zero the current populations of every solid cell in the bodies' tiles
template <typename S>
__global__ void k_zero_solid(S* __restrict__ fa, S* __restrict__ fb, const StepState* __restrict__ st,
                             const uint16_t* __restrict__ flags, const BodyDev* __restrict__ bodies, Lat lat) {
  using R = typename St<S>::R;
  const BodyDev& b = bodies[blockIdx.y];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b.sz) return;
  const unsigned u = (unsigned)t, L0 = (unsigned)b.L[0], L1 = (unsigned)b.L[1];
  const unsigned r = u / L0;
  const int gx = wrapi_near(b.o[0] + (int)(u - r * L0), lat.nx), gy = wrapi_near(b.o[1] + (int)(r % L1), lat.ny),
            gz = wrapi_near(b.o[2] + (int)(r / L1), lat.nz);
  const long long n = gx + (long long)lat.nx * (gy + (long long)lat.ny * gz);
  if (!(flags[n] & F_SOLID)) return;
  S* f = st->parity ? fb : fa;
#pragma unroll
  for (int i = 0; i < Q; ++i) St<S>::st(f, (size_t)i * lat.Ns + n, i, (R)0);
}

void launch_zero_solid(int prec, const Lat& lat, void* fa, void* fb, const StepState* st, const uint16_t* flags,
                       const BodyDev* bodies, int nb, int max_tile, cudaStream_t s) {
  if (!nb) return;
  dim3 grid((unsigned)((max_tile + 255) / 256), (unsigned)nb);
  if (prec == 0) k_zero_solid<double><<<grid, 256, 0, s>>>((double*)fa, (double*)fb, st, flags, bodies, lat);
  else if (prec == 1) k_zero_solid<float><<<grid, 256, 0, s>>>((float*)fa, (float*)fb, st, flags, bodies, lat);
  else k_zero_solid<__half><<<grid, 256, 0, s>>>((__half*)fa, (__half*)fb, st, flags, bodies, lat);
}

// ---- launchers -------------------------------------------------------------------------------
static int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

unsigned lbm_blocks(const Lat& lat) {
  const long long need = (lat.N + 255) / 256;
  const long long cap = 4LL * sm_count();  // a few resident blocks per SM, grid-stride beyond
  return (unsigned)(need < cap ? need : cap);
}

// Fused bulk pass: blocks of 32 x ty consumer columns (ty = 4 or 8) and as many producer threads,
// marching tz planes along z.
static int fused_min_blocks(int prec, int ty) {
  // resident blocks per SM asked of the compiler: 64 registers per thread for FP32 / binary16
  // storage, 128 for FP64
  const int thr = 2 * 32 * ty;
  return (prec == 0 ? 32768 : 65536) / (64 * thr);
}

// z extent of a fused block: enough blocks for `waves` full waves of resident blocks
int fused_tz(const Lat& lat, int prec, int ty, int waves) {
  const long long cols = (long long)((lat.nx + 31) / 32) * ((lat.ny + ty - 1) / ty);
  const long long slots = (long long)fused_min_blocks(prec, ty) * sm_count() * waves;
  long long nzc = (slots + cols - 1) / cols;
  if (nzc < 1) nzc = 1;
  if (nzc > lat.nz) nzc = lat.nz;
  return (int)((lat.nz + nzc - 1) / nzc);
}

template <typename S, int TY, int MINB>
static void fused_t(const Lat& lat, void* fa, void* fb, const uint16_t* flags, const BodyDev* bodies,
                    double* mass_part, const StepState* st, double* diag_rho, double* diag_vel, const PhysParams& pp,
                    int tz, cudaStream_t s) {
  const dim3 grid((lat.nx + 31) / 32, (lat.ny + TY - 1) / TY, (lat.nz + tz - 1) / tz);
  k_fused<S, 32, TY, TY, MINB><<<grid, 2 * 32 * TY, 0, s>>>((S*)fa, (S*)fb, flags, bodies, mass_part, st, diag_rho,
                                                           diag_vel, lat, pp, tz);
}

void launch_lbm_fused(int prec, const Lat& lat, void* fa, void* fb, const uint16_t* flags, const BodyDev* bodies,
                      double* mass_part, StepState* st, double* diag_rho, double* diag_vel, const PhysParams& pp,
                      int tz, int ty, cudaStream_t s) {
  if (ty == 4) {
    if (prec == 0) fused_t<double, 4, 2>(lat, fa, fb, flags, bodies, mass_part, st, diag_rho, diag_vel, pp, tz, s);
    else if (prec == 1) fused_t<float, 4, 4>(lat, fa, fb, flags, bodies, mass_part, st, diag_rho, diag_vel, pp, tz, s);
    else fused_t<__half, 4, 4>(lat, fa, fb, flags, bodies, mass_part, st, diag_rho, diag_vel, pp, tz, s);
  } else {
    if (prec == 0) fused_t<double, 8, 1>(lat, fa, fb, flags, bodies, mass_part, st, diag_rho, diag_vel, pp, tz, s);
    else if (prec == 1) fused_t<float, 8, 2>(lat, fa, fb, flags, bodies, mass_part, st, diag_rho, diag_vel, pp, tz, s);
    else fused_t<__half, 8, 2>(lat, fa, fb, flags, bodies, mass_part, st, diag_rho, diag_vel, pp, tz, s);
  }
}

void launch_density_tiles(int prec, const Lat& lat, const void* fa, const void* fb, const StepState* st,
                          const uint16_t* flags, const BodyDev* bodies, int nb, int max_tile, void* psi,
                          void* psi_b, const PhysParams& pp, cudaStream_t s) {
  if (!nb) return;
  const dim3 grid((unsigned)((max_tile + 255) / 256), (unsigned)nb);
  if (prec == 0)
    k_density_tiles<double><<<grid, 256, 0, s>>>((const double*)fa, (const double*)fb, st, flags, bodies,
                                                 (double*)psi, (double*)psi_b, lat, pp.rho0, pp.rho0_f);
  else if (prec == 1)
    k_density_tiles<float><<<grid, 256, 0, s>>>((const float*)fa, (const float*)fb, st, flags, bodies, (float*)psi,
                                                (float*)psi_b, lat, pp.rho0, pp.rho0_f);
  else
    k_density_tiles<__half><<<grid, 256, 0, s>>>((const __half*)fa, (const __half*)fb, st, flags, bodies,
                                                 (float*)psi, (float*)psi_b, lat, pp.rho0, pp.rho0_f);
}

template <typename S>
static void lbm_step_t(const Lat& lat, S* fa, S* fb, const uint16_t* flags, void* psi, void* psi_b,
                       const BodyDev* bodies, double* mass_part, unsigned blocks, StepState* st, double* diag_rho,
                       double* diag_vel, const PhysParams& pp, void* nbuf, const int* blist, cudaStream_t s,
                       int phases) {
  using R = typename St<S>::R;
  // `blocks` carries the x extent of the 128-thread blocks (32, 64 or 128)
  const int bx = blocks == 64 || blocks == 128 ? (int)blocks : 32, by = 128 / bx;
  const dim3 blk(bx, by, 1);
  const dim3 grid((lat.nx + bx - 1) / bx, (lat.ny + by - 1) / by, lat.nz);
  if (phases & 1)
    k_density<S><<<grid, blk, 0, s>>>(fa, fb, st, flags, bodies, (R*)psi, (R*)psi_b, lat, pp.rho0, pp.rho0_f);
  if (phases & 2)
    k_collide<S><<<grid, blk, 0, s>>>(fa, fb, flags, (const R*)psi, bodies, mass_part, st, diag_rho, diag_vel, lat,
                                      pp, (RhoPsi<R>*)nbuf);
  if ((phases & 4) && blist)
    k_collide_near<S><<<std::max(1, 2 * sm_count() / g_launch_share), 128, 0, s>>>(
        fa, fb, flags, (const R*)psi, (const R*)psi_b, bodies, mass_part, st, diag_rho, diag_vel, blist, lat, pp,
        (RhoPsi<R>*)nbuf);
}

void launch_lbm_step(int prec, const Lat& lat, void* fa, void* fb, const uint16_t* flags, void* psi, void* psi_b,
                     const BodyDev* bodies, double* mass_part, unsigned blocks, StepState* st, double* diag_rho,
                     double* diag_vel, const PhysParams& pp, void* nbuf, const int* blist, cudaStream_t s,
                     int phases) {
  if (prec == 0)
    lbm_step_t<double>(lat, (double*)fa, (double*)fb, flags, psi, psi_b, bodies, mass_part, blocks, st, diag_rho,
                       diag_vel, pp, nbuf, blist, s, phases);
  else if (prec == 1)
    lbm_step_t<float>(lat, (float*)fa, (float*)fb, flags, psi, psi_b, bodies, mass_part, blocks, st, diag_rho,
                      diag_vel, pp, nbuf, blist, s, phases);
  else
    lbm_step_t<__half>(lat, (__half*)fa, (__half*)fb, flags, psi, psi_b, bodies, mass_part, blocks, st, diag_rho,
                       diag_vel, pp, nbuf, blist, s, phases);
}

// Accumulating pass: blocks of 32 x ty threads (ty = 8 or 16) marching sz planes. Resident blocks
// per SM asked of the compiler: 64 registers per thread for FP32 storage, 80 for binary16, 128 for
// FP64.
static int acc_min_blocks(int prec, int ty) {
  const int regs = prec == 0 ? 128 : (prec == 1 ? 64 : 80);
  return std::max(1, 65536 / (regs * 32 * ty));
}

template <typename S, int TY>
static size_t acc_smem() {
  return (size_t)2 * (Q - 1) * 32 * TY * sizeof(typename St<S>::R);
}

// z extent of the accumulating pass's regions. A block marches its whole region, so the pass takes
// (waves of resident blocks) x (planes per region); the regions' edge planes add fix-up work. The
// extent minimises waves x planes + EDGE x (edge planes per resident block), over at most `waves`
// x 4 waves (EDGE: a fix-up plane costs about a fifth of a marched plane).
int acc_sz(const Lat& lat, int prec, int ty, int waves) {
  const long long cols = (long long)((lat.nx + 31) / 32) * ((lat.ny + ty - 1) / ty);
  const long long slots = (long long)acc_min_blocks(prec, ty) * sm_count();
  const double EDGE = 0.2;
  int best = lat.nz;
  double best_cost = 1e300;
  for (int sz = 1; sz <= lat.nz; ++sz) {
    const long long nzc = (lat.nz + sz - 1) / sz;
    if (sz < lat.nz && nzc * cols > slots * waves * 4) continue;
    const long long w = (nzc * cols + slots - 1) / slots;
    const double cost = (double)(w * sz) + EDGE * 2.0 * (double)(nzc * cols) / (double)slots;
    if (cost < best_cost) {
      best_cost = cost;
      best = sz;
    }
  }
  return best;
}

template <typename S, int TY, int MINB>
static cudaError_t acc_t(const Lat& lat, void* fa, void* fb, const uint16_t* flags, void* psi_a, void* psi_b,
                         void* rhop, const BodyDev* bodies, double* mass_part, StepState* st, double* diag_rho,
                         double* diag_vel, const PhysParams& pp, int sz, cudaStream_t s) {
  using R = typename St<S>::R;
  const size_t smem = acc_smem<S, TY>();
  // nz = 0: set the kernel's dynamic shared-memory limit (outside any stream capture) and return
  if (lat.nz <= 0)
    return cudaFuncSetAttribute(k_collide_acc<S, TY, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const dim3 grid((lat.nx + 31) / 32, (lat.ny + TY - 1) / TY, (lat.nz + sz - 1) / sz);
  k_collide_acc<S, TY, MINB><<<grid, 32 * TY, smem, s>>>((S*)fa, (S*)fb, flags, (R*)psi_a, (R*)psi_b, (R*)rhop,
                                                         bodies, mass_part, st, diag_rho, diag_vel, lat, pp, sz);
  return cudaGetLastError();
}

cudaError_t launch_lbm_acc(int prec, const Lat& lat, void* fa, void* fb, const uint16_t* flags, void* psi_a,
                           void* psi_b, void* rhop, const BodyDev* bodies, double* mass_part, StepState* st,
                           double* diag_rho, double* diag_vel, const PhysParams& pp, int ty, int sz,
                           cudaStream_t s) {
#define CBL_ACC(S, TY, MINB) \
  acc_t<S, TY, MINB>(lat, fa, fb, flags, psi_a, psi_b, rhop, bodies, mass_part, st, diag_rho, diag_vel, pp, sz, s)
  if (ty == 16) {
    if (prec == 0) return CBL_ACC(double, 16, 1);
    if (prec == 1) return CBL_ACC(float, 16, 2);
    return CBL_ACC(__half, 16, 1);
  }
  if (prec == 0) return CBL_ACC(double, 8, 2);
  if (prec == 1) return CBL_ACC(float, 8, 4);
  return CBL_ACC(__half, 8, 3);
#undef CBL_ACC
}

void launch_psi_fixup(int prec, const Lat& lat, const void* fa, const void* fb, void* psi_a, void* psi_b,
                      const void* rhop, const StepState* st, const PhysParams& pp, int ty, int sz, cudaStream_t s) {
  const AccGeom g = acc_geom(lat, ty, sz);
  const long long total = g.n1 + g.n2 + g.n3;
  const long long need = (total + 255) / 256, cap = 16LL * sm_count();
  const unsigned grid = (unsigned)std::max(1LL, std::min(need, cap));
  if (prec == 0)
    k_psi_fixup<double><<<grid, 256, 0, s>>>((const double*)fa, (const double*)fb, (double*)psi_a, (double*)psi_b,
                                             (const double*)rhop, st, lat, pp.rho0, pp.rho0_f, g);
  else if (prec == 1)
    k_psi_fixup<float><<<grid, 256, 0, s>>>((const float*)fa, (const float*)fb, (float*)psi_a, (float*)psi_b,
                                            (const float*)rhop, st, lat, pp.rho0, pp.rho0_f, g);
  else
    k_psi_fixup<__half><<<grid, 256, 0, s>>>((const __half*)fa, (const __half*)fb, (float*)psi_a, (float*)psi_b,
                                             (const float*)rhop, st, lat, pp.rho0, pp.rho0_f, g);
}

template <typename S>
static void boundary_t(const Lat& lat, const S* fa, const S* fb, const uint16_t* flags, const BodyDev* bodies,
                       double* acc, const int* blist, const StepState* st, const void* nbuf, double G,
                       cudaStream_t s) {
  using R = typename St<S>::R;
  // whole-lattice grid-stride rounds; the list length is only known on the device
  k_boundary<S><<<std::max(2, 8 * sm_count() / g_launch_share), 256, 0, s>>>(fa, fb, flags, bodies, acc, blist, st, (const RhoPsi<R>*)nbuf, lat, G,
                                                (float)G);
}

void launch_boundary(int prec, const Lat& lat, const void* fa, const void* fb, const uint16_t* flags,
                     const BodyDev* bodies, int nb, double* acc, const int* blist, const StepState* st,
                     const void* nbuf, double G, cudaStream_t s) {
  if (nb == 0) return;
  if (prec == 0)
    boundary_t<double>(lat, (const double*)fa, (const double*)fb, flags, bodies, acc, blist, st, nbuf, G, s);
  else if (prec == 1)
    boundary_t<float>(lat, (const float*)fa, (const float*)fb, flags, bodies, acc, blist, st, nbuf, G, s);
  else
    boundary_t<__half>(lat, (const __half*)fa, (const __half*)fb, flags, bodies, acc, blist, st, nbuf, G, s);
}

void launch_init_fluid(int prec, const Lat& lat, void* f, const uint16_t* flags, const double* rho, const double* u,
                       cudaStream_t s) {
  const int T = 256;
  const unsigned blocks = (unsigned)((lat.N + T - 1) / T);
  if (prec == 0) k_init_fluid<double><<<blocks, T, 0, s>>>((double*)f, flags, rho, u, lat);
  else if (prec == 1) k_init_fluid<float><<<blocks, T, 0, s>>>((float*)f, flags, rho, u, lat);
  else k_init_fluid<__half><<<blocks, T, 0, s>>>((__half*)f, flags, rho, u, lat);
}

void launch_refill(int prec, const Lat& lat, void* fa, void* fb, uint16_t* flags, const BodyDev* bodies, int nb,
                   int max_tile, StepState* st, int* blist, const double* arena, double member_thr, int* mbox,
                   int next, cudaStream_t s) {
  if (nb == 0) return;
  const int T = 256;
  dim3 grid((unsigned)((max_tile + T - 1) / T), (unsigned)nb);
  if (prec == 0)
    k_refill<double><<<grid, T, 0, s>>>((double*)fa, (double*)fb, flags, bodies, st, blist, lat, arena, member_thr,
                                        mbox, next);
  else if (prec == 1)
    k_refill<float><<<grid, T, 0, s>>>((float*)fa, (float*)fb, flags, bodies, st, blist, lat, arena, member_thr, mbox,
                                       next);
  else
    k_refill<__half><<<grid, T, 0, s>>>((__half*)fa, (__half*)fb, flags, bodies, st, blist, lat, arena, member_thr,
                                        mbox, next);
}

// Tile shapes of the persistent batch kernel (x, y, z cells; 128 threads per block).
void batch_tile(int cfg, int* t) {
  static const int T[BATCH_TILE_CFGS][3] = {{32, 4, 1}, {32, 4, 4}, {32, 4, 8}, {64, 2, 4}};
  const int k = cfg < 0 || cfg >= BATCH_TILE_CFGS ? 1 : cfg;
  for (int a = 0; a < 3; ++a) t[a] = T[k][a];
}

template <typename S, int TX, int TY, int TZ>
static int batch_occ() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_lbm<S, TX, TY, TZ>, TX * TY, 0);
  return nb;
}

template <typename S>
static int batch_occ_cfg(int cfg) {
  switch (cfg) {
    case 0: return batch_occ<S, 32, 4, 1>();
    case 2: return batch_occ<S, 32, 4, 8>();
    case 3: return batch_occ<S, 64, 2, 4>();
    default: return batch_occ<S, 32, 4, 4>();
  }
}

int batch_blocks_per_sm(int prec, int cfg) {
  return prec == 0 ? batch_occ_cfg<double>(cfg) : (prec == 1 ? batch_occ_cfg<float>(cfg) : batch_occ_cfg<__half>(cfg));
}

template <typename S, int TX, int TY, int TZ>
static cudaError_t batch_launch(const BatchInst* tab, int ninst, long long items, BatchCtl* ctl, int grid, int coop,
                                cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(TX * TY);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = coop ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_batch_lbm<S, TX, TY, TZ>, tab, ninst, items, ctl);
}

template <typename S>
static cudaError_t batch_launch_cfg(int cfg, const BatchInst* tab, int ninst, long long items, BatchCtl* ctl, int grid,
                                    int coop, cudaStream_t s) {
  switch (cfg) {
    case 0: return batch_launch<S, 32, 4, 1>(tab, ninst, items, ctl, grid, coop, s);
    case 2: return batch_launch<S, 32, 4, 8>(tab, ninst, items, ctl, grid, coop, s);
    case 3: return batch_launch<S, 64, 2, 4>(tab, ninst, items, ctl, grid, coop, s);
    default: return batch_launch<S, 32, 4, 4>(tab, ninst, items, ctl, grid, coop, s);
  }
}

cudaError_t launch_batch_lbm(int prec, int cfg, const BatchInst* tab, int ninst, long long items, BatchCtl* ctl,
                             int grid, int cooperative, cudaStream_t s) {
  if (prec == 0) return batch_launch_cfg<double>(cfg, tab, ninst, items, ctl, grid, cooperative, s);
  if (prec == 1) return batch_launch_cfg<float>(cfg, tab, ninst, items, ctl, grid, cooperative, s);
  return batch_launch_cfg<__half>(cfg, tab, ninst, items, ctl, grid, cooperative, s);
}

}  // namespace q19 / q27
}  // namespace cbl

#if CBL_Q == 19
// ---- one lattice-Boltzmann step with no allocation --------------------------------------------
// For callers that cannot allocate device memory (an allocator owned by another framework, a
// pre-reserved memory pool, a process that forbids cudaMalloc after start-up): the scratch this
// step needs (psi, an all-fluid flag field, the mass slots and the step state) lives in file-scope
// device arrays sized for CBL_NOALLOC_MAX_CELLS cells. Every GPU that loads the library holds them
// until the process exits.
namespace {
__device__ __align__(256) float g_na_psi[CBL_NOALLOC_MAX_CELLS];
__device__ __align__(256) uint16_t g_na_flags[CBL_NOALLOC_MAX_CELLS];
__device__ __align__(256) double g_na_mass[cbl::MASS_SLOTS];
__device__ __align__(256) cbl::StepState g_na_state;

// device addresses of the arrays, looked up with the calling device current
struct NaScratch {
  float* psi = nullptr;
  uint16_t* flags = nullptr;
  double* mass = nullptr;
  cbl::StepState* state = nullptr;
};

cudaError_t na_lookup(NaScratch& a) {
  cudaError_t e;
  if ((e = cudaGetSymbolAddress((void**)&a.psi, g_na_psi)) != cudaSuccess) return e;
  if ((e = cudaGetSymbolAddress((void**)&a.flags, g_na_flags)) != cudaSuccess) return e;
  if ((e = cudaGetSymbolAddress((void**)&a.mass, g_na_mass)) != cudaSuccess) return e;
  return cudaGetSymbolAddress((void**)&a.state, g_na_state);
}

__global__ void k_na_mass(const double* __restrict__ slots, double* __restrict__ out) {
  __shared__ double red[256];
  red[threadIdx.x] = slots[threadIdx.x];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}
}  // namespace

extern "C" cbl_status cbl_lbm_step_noalloc(const float* f_in, float* f_out, int nx, int ny, int nz, double tau,
                                           double G, double rho0, const double* ext_force, double* mass_out,
                                           void* stream) {
  using namespace cbl;
  using namespace cbl::q19;
  if (!f_in || !f_out) return CBL_ERR_ARG;
  if (nx < 4 || ny < 4 || nz < 4) return CBL_ERR_ARG;
  const long long N = (long long)nx * ny * nz;
  if (N > CBL_NOALLOC_MAX_CELLS) return CBL_ERR_ARG;
  if (!(tau > 0.5) || !(rho0 > 0) || !std::isfinite(tau) || !std::isfinite(G) || !std::isfinite(rho0)) return CBL_ERR_ARG;
  if (ext_force && !(std::isfinite(ext_force[0]) && std::isfinite(ext_force[1]) && std::isfinite(ext_force[2])))
    return CBL_ERR_ARG;
  // the two population arrays must not overlap (the step reads f_in while it writes f_out)
  const size_t pop = (size_t)Q * (size_t)N;
  if (f_out < f_in + pop && f_in < f_out + pop) return CBL_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // The arrays' device addresses are looked up on every call, with the calling device current
  // (cheap, and never stale after a device reset reloads the library's module). The first lookup on
  // a device may load the module: make the first call before any stream capture.
  NaScratch a;
  if (na_lookup(a) != cudaSuccess) return CBL_ERR_CUDA;
  // every call shares the arrays and they keep the last call's contents: clear what must start at
  // zero (all-fluid flags of this lattice, parity 0: read f_in and write f_out, no field record,
  // mass slots)
  if (cudaMemsetAsync(a.flags, 0, sizeof(uint16_t) * (size_t)N, s) != cudaSuccess) return CBL_ERR_CUDA;
  if (cudaMemsetAsync(a.state, 0, sizeof(StepState), s) != cudaSuccess) return CBL_ERR_CUDA;
  Lat lat;
  lat.nx = nx;
  lat.ny = ny;
  lat.nz = nz;
  lat.N = N;
  lat.Ns = N;  // the caller's arrays are packed
  PhysParams pp;
  memset(&pp, 0, sizeof(pp));
  pp.tau = tau;
  pp.G = G;
  pp.rho0 = rho0;
  for (int k = 0; k < 3; ++k) pp.ext[k] = ext_force ? ext_force[k] : 0.0;
  fill_float_params(pp);
  if (cudaMemsetAsync(a.mass, 0, sizeof(double) * MASS_SLOTS, s) != cudaSuccess) return CBL_ERR_CUDA;
  const dim3 blk(32, 4, 1);
  const dim3 grid((nx + 31) / 32, (ny + 3) / 4, nz);
  k_density<float><<<grid, blk, 0, s>>>(f_in, f_in, a.state, a.flags, nullptr, a.psi, nullptr, lat, rho0, (float)rho0);
  k_collide<float><<<grid, blk, 0, s>>>(const_cast<float*>(f_in), f_out, a.flags, a.psi, nullptr, a.mass, a.state,
                                        nullptr, nullptr, lat, pp, nullptr);
  if (mass_out) k_na_mass<<<1, 256, 0, s>>>(a.mass, mass_out);
  return cudaGetLastError() == cudaSuccess ? CBL_OK : CBL_ERR_CUDA;
}
#endif  // CBL_Q == 19 (no-allocation entry point)
