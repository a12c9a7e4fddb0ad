// FP64 CPU oracle for the combined multi-phase-field / lattice-Boltzmann time step
// (Schiedung, Tegeler, Medvedev, Varnik, "Simulation of Capillary-Driven Kinetics with
// Multi-Phase-Field and Lattice-Boltzmann Method", arXiv:1902.10432).
//
// TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the CUDA path is
// checked against. Only the test suite, the smoke check and the benchmark's CPU-baseline leg
// may load it. It shares no code, header, table or helper with the CUDA library.
//
// Everything is double precision. Every field is stored densely over the whole periodic
// lattice (one phase-field array per body), and every step follows the paper's order:
//   1. pull streaming with half-way bounce-back, moving-wall term g and the local mass
//      correction (Sec. 3.2.1 Eq. lb_streaming, Sec. 3.2.2 Eqs. lb_bounce_back,
//      lb_bounce_back_us, lb_bounce_back_mass), plus the momentum exchange on each body
//      (Sec. 3.2.2 Eq. solid_liquid_force);
//   2. moments and the pseudo-potential psi (Sec. 3.2.1, Sec. 3.2.3 Eq. mean_field_potential),
//      with solid cells acting as fluid of density varrho_B (Sec. 3.2.3, wetting);
//   3. Shan-Chen force (Eq. benzi_force) and its reaction on the bodies (Sec. 3.2.3);
//   4. BGK collision with Guo forcing (Eqs. lb_collision, distribution_eq, guo_forcing,
//      fluid_velocity);
//   5. solid-solid repulsion (Sec. 3.1.2 Eqs. soild_solid_potential, solid_solid_force);
//   6. rigid-body update (Sec. 3.1.1);
//   7. phase-field advection (Eq. phase_advection, directionally split, MC limiter, Sec. 3.3)
//      and multi-phase-field kinetics with volume restoration
//      (Eq. sim_proc_phase_field_dynamics and the Delta g definition in Sec. 3.3);
//   8. obstacle flags (fluid phase < 0.05, Sec. 3.2.2) and the cover refill /
//      uncover rule (Sec. 3.2.2).
// Where the paper is silent or garbled, the readings below are used (each marked READING).
//
// Parity status: functions are pinned by the tests in tests/test_oracle_*.py against closed
// forms, the paper's printed values and brute force. The solid-solid repulsion magnitude
// (e0, not given in the paper) and the MPF kinetics interface energies (sigma, not given)
// are parity unpinned in their magnitudes: only their structure (zero range, symmetry,
// stationarity of the flat profile) is pinned.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

typedef struct {
  int nx, ny, nz, q;           // lattice size, velocity set (19 or 27)
  double tau, G, rho0;         // BGK relaxation time, SC coupling, reference density
  double ext_force[3];         // uniform external force density on fluid cells
  int mpf_kinetics;            // 1: apply Eq. sim_proc_phase_field_dynamics after advection
  double mobility, eta;        // M_alpha_beta and interface width eta
  double sigma_sf, sigma_ss;   // interface energies solid-fluid, solid-solid (READING)
  double e0, rc;               // repulsion strength and range
  int nrep;                    // repulsion exponent n
  double solid_threshold;      // a cell is solid iff fluid phase < this (paper: 0.05)
  double member_threshold;     // repulsion body point iff phi_B >= this (READING: 0.5)
  int nthreads;                // OpenMP threads (0 = runtime default)
  int store_prec;              // storage model of the populations (analysis only, see round_store):
                               // 0 FP64 (the method), 1 FP32, 2 binary16 deviations from w_i
} orc_params;

}  // extern "C"

namespace {

struct Lattice {
  int Q = 0;
  int c[27][3];
  double w[27];
  int opp[27];
};

// Velocity sets. D3Q27 as printed in Sec. 3.2.1 (weights 8/27, 2/27, 1/54, 1/216);
// D3Q19 (READING: the textbook subset with |c|^2 <= 2, weights 1/3, 1/18, 1/36).
// The set is enumerated here, ordered by |c|^2, so the ordering is the oracle's own.
Lattice make_lattice(int Q) {
  Lattice L;
  L.Q = 0;
  for (int n2 = 0; n2 <= 3; ++n2) {
    for (int cz = -1; cz <= 1; ++cz)
      for (int cy = -1; cy <= 1; ++cy)
        for (int cx = -1; cx <= 1; ++cx) {
          int m = cx * cx + cy * cy + cz * cz;
          if (m != n2) continue;
          if (Q == 19 && m == 3) continue;
          double w;
          if (Q == 19) w = (m == 0) ? 1.0 / 3.0 : (m == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
          else w = (m == 0) ? 8.0 / 27.0 : (m == 1) ? 2.0 / 27.0 : (m == 2) ? 1.0 / 54.0 : 1.0 / 216.0;
          L.c[L.Q][0] = cx; L.c[L.Q][1] = cy; L.c[L.Q][2] = cz; L.w[L.Q] = w;
          L.Q++;
        }
  }
  for (int i = 0; i < L.Q; ++i)
    for (int j = 0; j < L.Q; ++j)
      if (L.c[j][0] == -L.c[i][0] && L.c[j][1] == -L.c[i][1] && L.c[j][2] == -L.c[i][2]) L.opp[i] = j;
  return L;
}

const double PI = 3.14159265358979323846;
// Numerical presence tolerance of a phase (READING): phi below it counts as absent and is set to 0
// at the clamp, phi above 1 - it is set to 1. Without it the limiter leaves ever smaller but
// non-zero values ahead of a moving front, and "phase present" (phi > 0) would hinge on rounding.
const double PHI_EPS = 1e-12;

struct Body {
  int shape;            // 0 sphere, 1 box
  double c0[3];         // nominal centre
  double radius;        // sphere radius of the phi = 1/2 surface
  double half[3];       // box half extents of the phi = 1/2 surface
  double q0[4];         // initial orientation (w, x, y, z)
  double rho_s;         // mass density rho_alpha
  double wet;           // wetting parameter varrho_B
  int fixed;
  int rot_lock = 0;     // bit c: the angular velocity component c is held at zero (see spans_lattice)
  double M = 0, Ibody[9] = {0};
  double X[3], Xprev[3], V[3] = {0, 0, 0}, W[3] = {0, 0, 0}, Q[4];
  double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};  // total force/torque of the last step
  double parts[18] = {0};  // momentum-exchange F,T | adhesion F,T | repulsion F,T
  double vol_ref = 0;
  std::vector<double> phi;  // dense, N
};

struct Oracle {
  orc_params p;
  Lattice L;
  int nx, ny, nz;
  long N;
  std::vector<double> f, fpre, rho, psi, vel;  // f: post-collision state, Q*N
  std::vector<uint8_t> solid;
  std::vector<int> owner;
  std::vector<Body> bodies;
  bool ready = false;
  long t = 0;
  long lost_refills = 0;

  long idx(int x, int y, int z) const { return (long)x + (long)nx * ((long)y + (long)ny * z); }
  static int wrap(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }
  void coords(long n, int& x, int& y, int& z) const {
    x = (int)(n % nx); long r = n / nx; y = (int)(r % ny); z = (int)(r / ny);
  }
  // minimum-image component: the representative of d modulo n in [-n/2, n/2). The IEEE remainder
  // is exact (d - k n with k the nearest integer to d / n, ties to even), so only the tie r = n/2
  // needs moving to -n/2; a non-finite d gives NaN.
  double mi(double d, int n) const {
    double r = std::remainder(d, (double)n);
    if (r >= 0.5 * n) r -= n;
    return r;
  }
  int dims(int d) const { return d == 0 ? nx : (d == 1 ? ny : nz); }
};

void cross(const double a[3], const double b[3], double r[3]) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

// Rotation matrix of a unit quaternion (w, x, y, z).
void quat_to_R(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

// Signed distance from a point (relative to the body centre) to the body surface,
// positive outside. Sphere: |r| - R. Box: exact box distance in the body frame.
double body_sdf(const Body& b, const double r[3]) {
  if (b.shape == 0) return std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) - b.radius;
  double R[9];
  quat_to_R(b.q0, R);
  double l[3], qv[3];
  for (int a = 0; a < 3; ++a) l[a] = R[0 + a] * r[0] + R[3 + a] * r[1] + R[6 + a] * r[2];  // R^T r
  for (int a = 0; a < 3; ++a) qv[a] = std::fabs(l[a]) - b.half[a];
  double o = 0, m = qv[0];
  for (int a = 0; a < 3; ++a) { double v = std::max(qv[a], 0.0); o += v * v; m = std::max(m, qv[a]); }
  return std::sqrt(o) + std::min(m, 0.0);
}

// Initial phase-field profile (READING of Sec. 3.1 with the interface width eta of Sec. 3.3):
// phi = 1/2 - 1/2 sin(pi d / eta) for |d| < eta/2, 1 inside, 0 outside. This is the profile
// for which I_alpha - I_beta vanishes in Eq. sim_proc_phase_field_dynamics.
double profile(double d, double eta) {
  if (d <= -0.5 * eta) return 1.0;
  if (d >= 0.5 * eta) return 0.0;
  return 0.5 - 0.5 * std::sin(PI * d / eta);
}

double feq(const Lattice& L, int i, double rho, const double u[3]) {
  // Eq. distribution_eq with the spurious sum dropped (READING), c_s^2 = 1/3.
  double cu = L.c[i][0] * u[0] + L.c[i][1] * u[1] + L.c[i][2] * u[2];
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return rho * L.w[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

// Body-point velocity, Eq. solid_velocity: u_B(x) = dX/dt + omega x (x - X_B).
void body_velocity(const Oracle& o, const Body& b, const double pos[3], const double Xref[3], double u[3]) {
  double r[3] = {o.mi(pos[0] - Xref[0], o.nx), o.mi(pos[1] - Xref[1], o.ny), o.mi(pos[2] - Xref[2], o.nz)};
  double wr[3];
  cross(b.W, r, wr);
  for (int a = 0; a < 3; ++a) u[a] = b.V[a] + wr[a];
}

int nthreads_of(const Oracle& o) {
#ifdef _OPENMP
  return o.p.nthreads > 0 ? o.p.nthreads : omp_get_max_threads();
#else
  (void)o;
  return 1;
#endif
}

// ---------------------------------------------------------------------------------------------
// Storage model (analysis only; not part of the paper's method, off by default). The CUDA library
// can store the populations in FP32, or as binary16 deviations h_i = f_i - w_i from the lattice
// weights. To separate what that storage costs from what its arithmetic costs, the oracle can round
// its stored populations the same way after every store (the collision and the cover refill) and
// otherwise stay FP64. Binary16 rounding is written out from the format: 11 significant bits for
// |h| >= 2^-14, a quantum of 2^-24 below, round to nearest even (std::nearbyint in the default
// rounding mode); the weights are rounded the same way first, so a zero population stays exact.
double round_binary16(double h) {
  const double a = std::fabs(h);
  if (a == 0.0) return h;
  if (a < 0x1p-14) return std::nearbyint(h * 0x1p24) * 0x1p-24;
  int e;
  std::frexp(a, &e);  // a = m 2^e, m in [0.5, 1): 11 significant bits are multiples of 2^(e - 11)
  return std::ldexp(std::nearbyint(std::ldexp(h, 11 - e)), e - 11);
}

void round_store(Oracle& o) {
  if (o.p.store_prec == 0) return;
  const int Q = o.L.Q;
  const long N = o.N;
  double wh[27];
  for (int i = 0; i < Q; ++i) wh[i] = round_binary16(o.L.w[i]);
#pragma omp parallel for schedule(static) num_threads(nthreads_of(o))
  for (long n = 0; n < N; ++n)
    for (int i = 0; i < Q; ++i) {
      double& f = o.f[(size_t)i * N + n];
      f = o.p.store_prec == 1 ? (double)(float)f : round_binary16((double)(float)(f - wh[i])) + wh[i];
    }
}

// ---------------------------------------------------------------------------------------------
// Flags: solid iff 1 - sum_B phi_B < threshold (Sec. 3.2.2); owner = argmax_B phi_B (READING,
// ties to the lower id). Also clamps each phi to [0, 1] and renormalises the solid sum to <= 1
// (READING: keeps the sum constraint of Sec. 3.1 after advection and kinetics).
void clamp_and_flag(Oracle& o, std::vector<uint8_t>& new_solid, std::vector<int>& new_owner) {
  long N = o.N;
  int nb = (int)o.bodies.size();
  new_solid.assign(N, 0);
  new_owner.assign(N, -1);
#pragma omp parallel for schedule(static) num_threads(nthreads_of(o))
  for (long n = 0; n < N; ++n) {
    double S = 0.0;
    for (int b = 0; b < nb; ++b) {
      double v = o.bodies[b].phi[n];
      v = std::min(1.0, std::max(0.0, v));
      if (v < PHI_EPS) v = 0.0;
      if (v > 1.0 - PHI_EPS) v = 1.0;
      o.bodies[b].phi[n] = v;
      S += v;
    }
    if (S > 1.0) {
      double S2 = 0.0;
      for (int b = 0; b < nb; ++b) {
        double v = o.bodies[b].phi[n] / S;
        o.bodies[b].phi[n] = v;
        S2 += v;
      }
      S = S2;
    }
    if (1.0 - S < o.p.solid_threshold) {
      new_solid[n] = 1;
      int best = 0;
      double bv = o.bodies[0].phi[n];
      for (int b = 1; b < nb; ++b)
        if (o.bodies[b].phi[n] > bv) { bv = o.bodies[b].phi[n]; best = b; }
      new_owner[n] = best;
    }
  }
}

// Mass, centre of mass and inertia from the phase field (READING; the paper gives only
// "mass density rho_alpha"): M = rho_a sum phi, X = sum x phi / sum phi,
// I = rho_a sum phi (|r|^2 1 - r r^T).
void body_props(Oracle& o, Body& b) {
  double s = 0, sx[3] = {0, 0, 0};
  for (long n = 0; n < o.N; ++n) {
    double v = b.phi[n];
    if (v == 0.0) continue;
    int x, y, z;
    o.coords(n, x, y, z);
    double r[3] = {o.mi(x - b.c0[0], o.nx), o.mi(y - b.c0[1], o.ny), o.mi(z - b.c0[2], o.nz)};
    s += v;
    for (int a = 0; a < 3; ++a) sx[a] += v * r[a];
  }
  double X[3];
  for (int a = 0; a < 3; ++a) {
    X[a] = b.c0[a] + sx[a] / s;
    int n = o.dims(a);
    X[a] = std::fmod(X[a], (double)n);
    if (X[a] < 0) X[a] += n;
  }
  double I[9] = {0};
  for (long n = 0; n < o.N; ++n) {
    double v = b.phi[n];
    if (v == 0.0) continue;
    int x, y, z;
    o.coords(n, x, y, z);
    double r[3] = {o.mi(x - X[0], o.nx), o.mi(y - X[1], o.ny), o.mi(z - X[2], o.nz)};
    double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) I[3 * a + c] += v * ((a == c ? rr : 0.0) - r[a] * r[c]);
  }
  b.M = b.rho_s * s;
  b.vol_ref = s;
  // body-frame inertia: I_body = R0^T I_world R0
  double R[9];
  quat_to_R(b.Q, R);
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      double acc = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) acc += R[3 * k + a] * (b.rho_s * I[3 * k + l]) * R[3 * l + c];
      b.Ibody[3 * a + c] = acc;
    }
  for (int a = 0; a < 3; ++a) { b.X[a] = X[a]; b.Xprev[a] = X[a]; }
}

void rasterize(Oracle& o, Body& b) {
  b.phi.assign(o.N, 0.0);
  for (long n = 0; n < o.N; ++n) {
    int x, y, z;
    o.coords(n, x, y, z);
    double r[3] = {o.mi(x - b.c0[0], o.nx), o.mi(y - b.c0[1], o.ny), o.mi(z - b.c0[2], o.nz)};
    b.phi[n] = profile(body_sdf(b, r), o.p.eta);
  }
}

// ---------------------------------------------------------------------------------------------
// Step part 1-4: streaming with bounce-back, moments, SC force, collision.
void lbm_step(Oracle& o) {
  const Lattice& L = o.L;
  const int Q = L.Q, nx = o.nx, ny = o.ny, nz = o.nz;
  const long N = o.N;
  const int nb = (int)o.bodies.size();
  // per z-plane partial sums of the body force parts, summed in plane order afterwards so the
  // result does not depend on the thread count
  std::vector<double> part((size_t)nz * nb * 12, 0.0);

  // 1. pull streaming + bounce-back + g + delta rho + momentum exchange
#pragma omp parallel for schedule(static) num_threads(nthreads_of(o))
  for (int z = 0; z < nz; ++z) {
    double* pz = nb ? &part[(size_t)z * nb * 12] : nullptr;
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long n = o.idx(x, y, z);
        if (o.solid[n]) {
          for (int i = 0; i < Q; ++i) o.fpre[(size_t)i * N + n] = 0.0;
          o.rho[n] = 0.0;
          continue;
        }
        bool link_solid[27];
        for (int i = 0; i < Q; ++i) {
          long s = o.idx(Oracle::wrap(x - L.c[i][0], nx), Oracle::wrap(y - L.c[i][1], ny),
                         Oracle::wrap(z - L.c[i][2], nz));
          link_solid[i] = (i != 0) && o.solid[s];
          o.fpre[(size_t)i * N + n] = link_solid[i] ? o.f[(size_t)L.opp[i] * N + n] : o.f[(size_t)i * N + s];
        }
        // density after streaming; the g terms below cancel in it because of delta rho
        double r = 0.0;
        for (int i = 0; i < Q; ++i) r += o.fpre[(size_t)i * N + n];
        o.rho[n] = r;
        double drho = 0.0;
        for (int i = 1; i < Q; ++i) {
          if (!link_solid[i]) continue;
          long s = o.idx(Oracle::wrap(x - L.c[i][0], nx), Oracle::wrap(y - L.c[i][1], ny),
                         Oracle::wrap(z - L.c[i][2], nz));
          int B = o.owner[s];
          const Body& b = o.bodies[B];
          double mid[3] = {x - 0.5 * L.c[i][0], y - 0.5 * L.c[i][1], z - 0.5 * L.c[i][2]};
          double uB[3];
          body_velocity(o, b, mid, b.X, uB);
          double cu = L.c[i][0] * uB[0] + L.c[i][1] * uB[1] + L.c[i][2] * uB[2];
          double g = 2.0 * r * L.w[i] * cu * 3.0;  // 2 rho w_i c_i.u_B / c_s^2
          double fbar = o.f[(size_t)L.opp[i] * N + n];
          o.fpre[(size_t)i * N + n] += g;
          drho -= g;  // READING: negative sum, so that the g terms add no mass
          // momentum exchange on B: -c_i (2 f*_opp(x) + g), arm at the link midpoint
          double dP[3];
          for (int a = 0; a < 3; ++a) dP[a] = -L.c[i][a] * (2.0 * fbar + g);
          double arm[3] = {o.mi(mid[0] - b.X[0], nx), o.mi(mid[1] - b.X[1], ny), o.mi(mid[2] - b.X[2], nz)};
          double dL[3];
          cross(arm, dP, dL);
          for (int a = 0; a < 3; ++a) { pz[B * 12 + a] += dP[a]; pz[B * 12 + 3 + a] += dL[a]; }
        }
        o.fpre[n] += drho;  // i = 0 is the rest population in this ordering
      }
  }

  // 2. pseudo-potential; solid cells carry the wetting density of their owner
#pragma omp parallel for schedule(static) num_threads(nthreads_of(o))
  for (long n = 0; n < N; ++n) {
    double r = o.solid[n] ? o.bodies[o.owner[n]].wet : o.rho[n];
    o.psi[n] = 1.0 - std::exp(-r / o.p.rho0);
  }

  // 3-4. SC force, adhesion reaction, Guo-forced BGK collision
  const double tau = o.p.tau, G = o.p.G;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(o))
  for (int z = 0; z < nz; ++z) {
    double* pz = nb ? &part[(size_t)z * nb * 12] : nullptr;
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long n = o.idx(x, y, z);
        if (o.solid[n]) {
          for (int i = 0; i < Q; ++i) o.f[(size_t)i * N + n] = 0.0;
          for (int a = 0; a < 3; ++a) o.vel[3 * n + a] = 0.0;
          continue;
        }
        double ps = o.psi[n];
        double sum[3] = {0, 0, 0};
        for (int i = 1; i < Q; ++i) {
          long m = o.idx(Oracle::wrap(x + L.c[i][0], nx), Oracle::wrap(y + L.c[i][1], ny),
                         Oracle::wrap(z + L.c[i][2], nz));
          double wp = L.w[i] * o.psi[m];
          for (int a = 0; a < 3; ++a) sum[a] += wp * L.c[i][a];
          if (o.solid[m]) {
            int B = o.owner[m];
            const Body& b = o.bodies[B];
            double fr[3];
            for (int a = 0; a < 3; ++a) fr[a] = G * ps * wp * L.c[i][a];  // reaction on the body
            double pos[3] = {(double)x + L.c[i][0], (double)y + L.c[i][1], (double)z + L.c[i][2]};
            double arm[3] = {o.mi(pos[0] - b.X[0], nx), o.mi(pos[1] - b.X[1], ny), o.mi(pos[2] - b.X[2], nz)};
            double tq[3];
            cross(arm, fr, tq);
            for (int a = 0; a < 3; ++a) { pz[B * 12 + 6 + a] += fr[a]; pz[B * 12 + 9 + a] += tq[a]; }
          }
        }
        double F[3];
        for (int a = 0; a < 3; ++a) F[a] = -G * ps * sum[a] + o.p.ext_force[a];
        double r = o.rho[n];
        double mom[3] = {0.5 * F[0], 0.5 * F[1], 0.5 * F[2]};
        for (int i = 0; i < Q; ++i) {
          double fi = o.fpre[(size_t)i * N + n];
          for (int a = 0; a < 3; ++a) mom[a] += L.c[i][a] * fi;
        }
        double v[3] = {0, 0, 0};
        if (r > 0.0)
          for (int a = 0; a < 3; ++a) v[a] = mom[a] / r;
        for (int a = 0; a < 3; ++a) o.vel[3 * n + a] = v[a];
        double pref = 1.0 - 0.5 / tau;
        for (int i = 0; i < Q; ++i) {
          double fi = o.fpre[(size_t)i * N + n];
          double cv = L.c[i][0] * v[0] + L.c[i][1] * v[1] + L.c[i][2] * v[2];
          double Fi = 0.0;
          for (int a = 0; a < 3; ++a) Fi += (3.0 * (L.c[i][a] - v[a]) + 9.0 * cv * L.c[i][a]) * F[a];
          Fi *= pref * L.w[i];
          o.f[(size_t)i * N + n] = fi - (fi - feq(L, i, r, v)) / tau + Fi;
        }
      }
  }

  for (int b = 0; b < nb; ++b) {
    double s[12] = {0};
    for (int z = 0; z < nz; ++z)
      for (int k = 0; k < 12; ++k) s[k] += part[((size_t)z * nb + b) * 12 + k];
    for (int k = 0; k < 12; ++k) o.bodies[b].parts[k] = s[k];
    for (int k = 12; k < 18; ++k) o.bodies[b].parts[k] = 0.0;
  }
}

// Step part 5: solid-solid repulsion, Eqs. soild_solid_potential / solid_solid_force.
// Body points: cells with phi_B >= member_threshold (READING). Each ordered pair (x_i in A,
// x_j in B, 0 < |x_i - x_j| < r_c) pushes A along (x_i - x_j) with magnitude
// e0 n / r_c |(d - r_c)/r_c|^(n-1); the torque arm is x_i - X_A.
void repulsion(Oracle& o) {
  const int nb = (int)o.bodies.size();
  if (nb < 2 || o.p.e0 == 0.0) return;
  const double rc = o.p.rc;
  const int R = (int)std::ceil(rc);
  std::vector<int> off;
  for (int dz = -R; dz <= R; ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        int d2 = dx * dx + dy * dy + dz * dz;
        if (d2 > 0 && (double)d2 < rc * rc) { off.push_back(dx); off.push_back(dy); off.push_back(dz); }
      }
  int noff = (int)off.size() / 3;
  for (int A = 0; A < nb; ++A) {
    Body& a = o.bodies[A];
    double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
    for (int B = 0; B < nb; ++B) {
      if (B == A) continue;
      const Body& b = o.bodies[B];
      for (long n = 0; n < o.N; ++n) {
        if (a.phi[n] < o.p.member_threshold) continue;
        int x, y, z;
        o.coords(n, x, y, z);
        for (int k = 0; k < noff; ++k) {
          int dx = off[3 * k], dy = off[3 * k + 1], dz = off[3 * k + 2];
          long m = o.idx(Oracle::wrap(x + dx, o.nx), Oracle::wrap(y + dy, o.ny), Oracle::wrap(z + dz, o.nz));
          if (b.phi[m] < o.p.member_threshold) continue;
          double d = std::sqrt((double)(dx * dx + dy * dy + dz * dz));
          double mag = o.p.e0 * o.p.nrep / rc * std::pow(std::fabs((d - rc) / rc), o.p.nrep - 1);
          double fv[3] = {-dx / d * mag, -dy / d * mag, -dz / d * mag};
          double arm[3] = {o.mi(x - a.X[0], o.nx), o.mi(y - a.X[1], o.ny), o.mi(z - a.X[2], o.nz)};
          double tq[3];
          cross(arm, fv, tq);
          for (int c = 0; c < 3; ++c) { F[c] += fv[c]; T[c] += tq[c]; }
        }
      }
    }
    for (int c = 0; c < 3; ++c) { a.parts[12 + c] = F[c]; a.parts[15 + c] = T[c]; }
  }
}

// Step part 6: rigid-body update (Sec. 3.1.1). READING (integrator not given): semi-implicit
// Euler with dt = 1: V += F/M, X += V, omega += I_w^-1 T with I_w = R I_body R^T,
// q <- normalize(exp(omega/2) q).
void integrate_body(Oracle& o, Body& b) {
  for (int a = 0; a < 3; ++a) {
    b.F[a] = b.parts[a] + b.parts[6 + a] + b.parts[12 + a];
    b.T[a] = b.parts[3 + a] + b.parts[9 + a] + b.parts[15 + a];
    b.Xprev[a] = b.X[a];
  }
  if (b.fixed) {
    for (int a = 0; a < 3; ++a) { b.V[a] = 0; b.W[a] = 0; }
    return;
  }
  for (int a = 0; a < 3; ++a) {
    b.V[a] += b.F[a] / b.M;
    double x = b.X[a] + b.V[a];
    int n = o.dims(a);
    x = std::fmod(x, (double)n);
    if (x < 0) x += n;
    b.X[a] = x;
  }
  double R[9], Iw[9];
  quat_to_R(b.Q, R);
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      double acc = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) acc += R[3 * a + k] * b.Ibody[3 * k + l] * R[3 * c + l];
      Iw[3 * a + c] = acc;
    }
  // solve Iw dw = T by Cramer's rule
  double det = Iw[0] * (Iw[4] * Iw[8] - Iw[5] * Iw[7]) - Iw[1] * (Iw[3] * Iw[8] - Iw[5] * Iw[6]) +
               Iw[2] * (Iw[3] * Iw[7] - Iw[4] * Iw[6]);
  double inv[9];
  inv[0] = (Iw[4] * Iw[8] - Iw[5] * Iw[7]) / det;
  inv[1] = (Iw[2] * Iw[7] - Iw[1] * Iw[8]) / det;
  inv[2] = (Iw[1] * Iw[5] - Iw[2] * Iw[4]) / det;
  inv[3] = (Iw[5] * Iw[6] - Iw[3] * Iw[8]) / det;
  inv[4] = (Iw[0] * Iw[8] - Iw[2] * Iw[6]) / det;
  inv[5] = (Iw[2] * Iw[3] - Iw[0] * Iw[5]) / det;
  inv[6] = (Iw[3] * Iw[7] - Iw[4] * Iw[6]) / det;
  inv[7] = (Iw[1] * Iw[6] - Iw[0] * Iw[7]) / det;
  inv[8] = (Iw[0] * Iw[4] - Iw[1] * Iw[3]) / det;
  for (int a = 0; a < 3; ++a) b.W[a] += inv[3 * a] * b.T[0] + inv[3 * a + 1] * b.T[1] + inv[3 * a + 2] * b.T[2];
  for (int a = 0; a < 3; ++a)
    if (b.rot_lock >> a & 1) b.W[a] = 0.0;
  double wn = std::sqrt(b.W[0] * b.W[0] + b.W[1] * b.W[1] + b.W[2] * b.W[2]);
  if (wn > 0) {
    double h = 0.5 * wn, s = std::sin(h) / wn;
    double dq[4] = {std::cos(h), b.W[0] * s, b.W[1] * s, b.W[2] * s};
    const double* q = b.Q;
    double nq[4] = {dq[0] * q[0] - dq[1] * q[1] - dq[2] * q[2] - dq[3] * q[3],
                    dq[0] * q[1] + dq[1] * q[0] + dq[2] * q[3] - dq[3] * q[2],
                    dq[0] * q[2] - dq[1] * q[3] + dq[2] * q[0] + dq[3] * q[1],
                    dq[0] * q[3] + dq[1] * q[2] - dq[2] * q[1] + dq[3] * q[0]};
    double qn = std::sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
    for (int a = 0; a < 4; ++a) b.Q[a] = nq[a] / qn;
  }
}

// Monotonized-central limited slope (van Leer 1977): minmod(2 dm, (dm + dp)/2, 2 dp).
double mc_slope(double dm, double dp) {
  if (dm * dp <= 0.0) return 0.0;
  double s = std::min(std::min(2.0 * std::fabs(dm), 0.5 * std::fabs(dm + dp)), 2.0 * std::fabs(dp));
  return dm > 0 ? s : -s;
}

// Step part 7a: one conservative 1D sweep of d(phi)/dt = -u . grad(phi) along axis d
// (READING of the garbled sign of Eq. phase_advection). Face value: upwind cell value plus
// half of (1 - |u|) times its MC-limited slope; face velocity: the d-component of u_B at the
// face centre, using the new V and omega and the pre-update centre of mass.
void sweep(Oracle& o, Body& b, int d, std::vector<double>& out) {
  const int nx = o.nx, ny = o.ny, nz = o.nz;
  const long N = o.N;
  std::vector<double> flux(N);
  const std::vector<double>& phi = b.phi;
  int e[3] = {d == 0, d == 1, d == 2};
#pragma omp parallel for schedule(static) num_threads(nthreads_of(o))
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        // face between cell i = (x,y,z) and i + e_d
        auto at = [&](int k) {
          return phi[o.idx(Oracle::wrap(x + k * e[0], nx), Oracle::wrap(y + k * e[1], ny),
                           Oracle::wrap(z + k * e[2], nz))];
        };
        double pm1 = at(-1), p0 = at(0), p1 = at(1), p2 = at(2);
        double pos[3] = {x + 0.5 * e[0], y + 0.5 * e[1], z + 0.5 * e[2]};
        double u[3];
        body_velocity(o, b, pos, b.Xprev, u);
        double uf = u[d];
        double face;
        if (uf >= 0.0) face = p0 + 0.5 * (1.0 - uf) * mc_slope(p0 - pm1, p1 - p0);
        else face = p1 - 0.5 * (1.0 + uf) * mc_slope(p1 - p0, p2 - p1);
        flux[o.idx(x, y, z)] = uf * face;
      }
  out.resize(N);
#pragma omp parallel for schedule(static) num_threads(nthreads_of(o))
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long n = o.idx(x, y, z);
        long m = o.idx(Oracle::wrap(x - e[0], nx), Oracle::wrap(y - e[1], ny), Oracle::wrap(z - e[2], nz));
        out[n] = phi[n] - (flux[n] - flux[m]);
      }
}

void advect(Oracle& o) {
  std::vector<double> tmp;
  for (Body& b : o.bodies) {
    bool still = b.V[0] == 0 && b.V[1] == 0 && b.V[2] == 0 && b.W[0] == 0 && b.W[1] == 0 && b.W[2] == 0;
    if (still) continue;  // every face flux is exactly zero
    for (int d = 0; d < 3; ++d) {
      sweep(o, b, d, tmp);
      b.phi.swap(tmp);
    }
  }
}

// Step part 7b: Eq. sim_proc_phase_field_dynamics, one explicit Euler step (dt = 1).
// READINGS: N = number of phases active at the cell (phi > PHI_EPS at the cell or one of its 6
// face neighbours; the fluid phase is 1 - sum of solid phases); sigma between a solid and the
// fluid is sigma_sf, between two solids sigma_ss; the volume term (pi^2/(4 eta)) Delta g_ab
// equals D_a - D_b with D_B = (V_B(0) - sum phi_B) / #{0 < phi_B < 1} for a solid and D = 0 for
// the fluid, and is applied only where 0 < phi_a < 1 (both "0 <" and "< 1" with the PHI_EPS
// tolerance); 7-point Laplacian.
void kinetics(Oracle& o) {
  const int nb = (int)o.bodies.size();
  if (nb == 0) return;
  const long N = o.N;
  const int nx = o.nx, ny = o.ny, nz = o.nz;
  const double eta = o.p.eta, k2 = PI * PI / (eta * eta), M = o.p.mobility;
  std::vector<double> D(nb + 1, 0.0);
  for (int b = 0; b < nb; ++b) {
    double s = 0;
    long cnt = 0;
    for (long n = 0; n < N; ++n) {
      double v = o.bodies[b].phi[n];
      s += v;
      if (v > PHI_EPS && v < 1.0 - PHI_EPS) cnt++;
    }
    D[b] = cnt ? (o.bodies[b].vol_ref - s) / (double)cnt : 0.0;
  }
  D[nb] = 0.0;  // fluid
  std::vector<double> S(N, 0.0);
  for (int b = 0; b < nb; ++b)
    for (long n = 0; n < N; ++n) S[n] += o.bodies[b].phi[n];
  std::vector<std::vector<double>> out(nb);
  for (int b = 0; b < nb; ++b) out[b] = o.bodies[b].phi;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(o))
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long n = o.idx(x, y, z);
        long nbr[6] = {o.idx(Oracle::wrap(x + 1, nx), y, z), o.idx(Oracle::wrap(x - 1, nx), y, z),
                       o.idx(x, Oracle::wrap(y + 1, ny), z), o.idx(x, Oracle::wrap(y - 1, ny), z),
                       o.idx(x, y, Oracle::wrap(z + 1, nz)), o.idx(x, y, Oracle::wrap(z - 1, nz))};
        // active phases: solids ascending, then the fluid (index nb)
        int act[64];
        int na = 0;
        for (int b = 0; b < nb && na < 63; ++b) {
          const std::vector<double>& ph = o.bodies[b].phi;
          bool on = ph[n] > PHI_EPS;
          for (int k = 0; k < 6 && !on; ++k) on = ph[nbr[k]] > PHI_EPS;
          if (on) act[na++] = b;
        }
        bool fl = S[n] < 1.0 - PHI_EPS;
        for (int k = 0; k < 6 && !fl; ++k) fl = S[nbr[k]] < 1.0 - PHI_EPS;
        if (fl) act[na++] = nb;
        if (na <= 1) continue;
        double I[64];
        for (int k = 0; k < na; ++k) {
          int a = act[k];
          double c0, lap = 0.0;
          if (a < nb) {
            const std::vector<double>& ph = o.bodies[a].phi;
            c0 = ph[n];
            for (int j = 0; j < 6; ++j) lap += ph[nbr[j]];
          } else {
            c0 = 1.0 - S[n];
            for (int j = 0; j < 6; ++j) lap += 1.0 - S[nbr[j]];
          }
          lap -= 6.0 * c0;
          I[k] = lap + k2 * c0;
        }
        auto sig = [&](int a, int b) {
          return (a == nb || b == nb) ? o.p.sigma_sf : o.p.sigma_ss;
        };
        for (int ka = 0; ka < na; ++ka) {
          int a = act[ka];
          if (a == nb) continue;  // the fluid phase is implicit
          double pa = o.bodies[a].phi[n];
          bool in_if = pa > PHI_EPS && pa < 1.0 - PHI_EPS;
          double rate = 0.0;
          for (int kb = 0; kb < na; ++kb) {
            if (kb == ka) continue;
            int b = act[kb];
            double term = sig(a, b) * (I[ka] - I[kb]);
            for (int kg = 0; kg < na; ++kg) {
              if (kg == ka || kg == kb) continue;
              int g = act[kg];
              term += (sig(b, g) - sig(a, g)) * I[kg];
            }
            if (in_if) term += D[a] - D[b];
            rate += M / na * term;
          }
          out[a][n] = pa + rate;
        }
      }
  for (int b = 0; b < nb; ++b) o.bodies[b].phi.swap(out[b]);
}

// Step part 8: new flags, cover refill and uncover (Sec. 3.2.2). READING: a newly solid
// node n hands f_eq(rho_n, u_n) / |N_F| to each fluid face neighbour (R_A = dx); if it has
// none, to each fluid node within sqrt(3); rho_n and u_n are the plain moments of its
// populations. Newly fluid nodes start from zero populations.
void flags_and_refill(Oracle& o) {
  std::vector<uint8_t> ns;
  std::vector<int> nown;
  clamp_and_flag(o, ns, nown);
  const Lattice& L = o.L;
  const int Q = L.Q;
  const long N = o.N;
  for (long n = 0; n < N; ++n) {
    if (!(ns[n] && !o.solid[n])) continue;
    int x, y, z;
    o.coords(n, x, y, z);
    double r = 0, mom[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
      double fi = o.f[(size_t)i * N + n];
      r += fi;
      for (int a = 0; a < 3; ++a) mom[a] += L.c[i][a] * fi;
    }
    double u[3] = {0, 0, 0};
    if (r > 0)
      for (int a = 0; a < 3; ++a) u[a] = mom[a] / r;
    std::vector<long> nf;
    for (int pass = 0; pass < 2 && nf.empty(); ++pass)
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int d2 = dx * dx + dy * dy + dz * dz;
            if (d2 == 0 || (pass == 0 && d2 > 1)) continue;
            long m = o.idx(Oracle::wrap(x + dx, o.nx), Oracle::wrap(y + dy, o.ny), Oracle::wrap(z + dz, o.nz));
            if (!ns[m]) nf.push_back(m);
          }
    if (nf.empty()) {
      o.lost_refills++;
    } else {
      double inv = 1.0 / (double)nf.size();
      for (long m : nf)
        for (int i = 0; i < Q; ++i) o.f[(size_t)i * N + m] += feq(L, i, r, u) * inv;
    }
    for (int i = 0; i < Q; ++i) o.f[(size_t)i * N + n] = 0.0;
  }
  o.solid.swap(ns);
  o.owner.swap(nown);
}

}  // namespace

extern "C" {

void* orc_create(const orc_params* p) {
  if (!p || p->nx <= 0 || p->ny <= 0 || p->nz <= 0 || (p->q != 19 && p->q != 27) || !(p->tau > 0.5))
    return nullptr;
  Oracle* o = new Oracle();
  o->p = *p;
  o->L = make_lattice(p->q);
  o->nx = p->nx; o->ny = p->ny; o->nz = p->nz;
  o->N = (long)p->nx * p->ny * p->nz;
  return o;
}

void orc_destroy(void* h) { delete (Oracle*)h; }

// A body whose phi support (surface + eta/2) covers the whole periodic length of the lattice
// along an axis is infinite along that axis: the plates of the planar bridge of Sec. 2.1, whose
// length L is the lattice length under periodic boundaries. READING (the paper does not say how
// such a body turns): it may turn only about that axis, since a turn about any other axis would
// break its periodicity (and the lever arm at the periodic seam is not defined); the rigid-body
// update holds the other angular-velocity components at zero. Returns the bit mask of the held
// components.
int rotation_lock(const Oracle& o, const Body& b) {
  double h[3];
  if (b.shape == 0) {
    for (int a = 0; a < 3; ++a) h[a] = b.radius;
  } else {
    double R[9];
    quat_to_R(b.q0, R);
    for (int a = 0; a < 3; ++a)
      h[a] = std::fabs(R[3 * a]) * b.half[0] + std::fabs(R[3 * a + 1]) * b.half[1] + std::fabs(R[3 * a + 2]) * b.half[2];
  }
  int lock = 0;
  for (int a = 0; a < 3; ++a)
    if (2.0 * (h[a] + 0.5 * o.p.eta) >= (double)o.dims(a))
      for (int c = 0; c < 3; ++c)
        if (c != a) lock |= 1 << c;
  return lock;
}

int orc_add_body(void* h, int shape, const double* center, double radius, const double* half,
                 const double* quat, double mass_density, double wetting_rho, int fixed) {
  Oracle* o = (Oracle*)h;
  if (o->ready) return -1;
  Body b;
  b.shape = shape;
  for (int a = 0; a < 3; ++a) { b.c0[a] = center[a]; b.half[a] = half ? half[a] : 0.0; }
  b.radius = radius;
  double qn = 1.0;
  if (quat) qn = std::sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
  for (int a = 0; a < 4; ++a) b.q0[a] = quat ? quat[a] / qn : (a == 0 ? 1.0 : 0.0);
  for (int a = 0; a < 4; ++a) b.Q[a] = b.q0[a];
  b.rho_s = mass_density;
  b.wet = wetting_rho;
  b.fixed = fixed;
  b.rot_lock = rotation_lock(*o, b);
  rasterize(*o, b);
  o->bodies.push_back(std::move(b));
  return (int)o->bodies.size() - 1;
}

// rho_init/u_init: per-cell density and velocity (u may be NULL for rest). Solid cells get 0.
int orc_init_fluid_fields(void* h, const double* rho_init, const double* u_init) {
  Oracle* o = (Oracle*)h;
  const long N = o->N;
  const int Q = o->L.Q;
  o->f.assign((size_t)Q * N, 0.0);
  o->fpre.assign((size_t)Q * N, 0.0);
  o->rho.assign(N, 0.0);
  o->psi.assign(N, 0.0);
  o->vel.assign(3 * N, 0.0);
  o->solid.assign(N, 0);
  o->owner.assign(N, -1);
  if (!o->bodies.empty()) {
    std::vector<uint8_t> ns;
    std::vector<int> nown;
    clamp_and_flag(*o, ns, nown);
    o->solid.swap(ns);
    o->owner.swap(nown);
    for (Body& b : o->bodies) body_props(*o, b);
  }
  for (long n = 0; n < N; ++n) {
    if (o->solid[n]) continue;
    double u[3] = {0, 0, 0};
    if (u_init)
      for (int a = 0; a < 3; ++a) u[a] = u_init[3 * n + a];
    for (int i = 0; i < Q; ++i) o->f[(size_t)i * N + n] = feq(o->L, i, rho_init[n], u);
    o->rho[n] = rho_init[n];
    for (int a = 0; a < 3; ++a) o->vel[3 * n + a] = u[a];
  }
  o->ready = true;
  o->t = 0;
  return 0;
}

// Sharp liquid/vapour initial state: rho_l where mask != 0, rho_v elsewhere, at rest.
int orc_init_fluid(void* h, double rho_l, double rho_v, const unsigned char* mask) {
  Oracle* o = (Oracle*)h;
  std::vector<double> r(o->N);
  for (long n = 0; n < o->N; ++n) r[n] = (mask && mask[n]) ? rho_l : rho_v;
  return orc_init_fluid_fields(h, r.data(), nullptr);
}

int orc_step(void* h, int nsteps) {
  Oracle* o = (Oracle*)h;
  if (!o->ready) return -1;
  for (int s = 0; s < nsteps; ++s) {
    lbm_step(*o);
    round_store(*o);
    repulsion(*o);
    for (Body& b : o->bodies) integrate_body(*o, b);
    if (!o->bodies.empty()) {
      advect(*o);
      if (o->p.mpf_kinetics) kinetics(*o);
      flags_and_refill(*o);
      round_store(*o);
    }
    o->t++;
  }
  return 0;
}

long orc_num_cells(void* h) { return ((Oracle*)h)->N; }
long orc_time(void* h) { return ((Oracle*)h)->t; }
long orc_lost_refills(void* h) { return ((Oracle*)h)->lost_refills; }
int orc_num_bodies(void* h) { return (int)((Oracle*)h)->bodies.size(); }

// Fluid density and velocity of the last collision (0 on solid cells); fluid phase 1 - sum phi.
void orc_read_fields(void* h, double* rho, double* vel, double* phi_fluid) {
  Oracle* o = (Oracle*)h;
  for (long n = 0; n < o->N; ++n) {
    if (rho) rho[n] = o->solid[n] ? 0.0 : o->rho[n];
    if (vel)
      for (int a = 0; a < 3; ++a) vel[3 * n + a] = o->solid[n] ? 0.0 : o->vel[3 * n + a];
    if (phi_fluid) {
      double S = 0;
      for (const Body& b : o->bodies) S += b.phi[n];
      phi_fluid[n] = 1.0 - S;
    }
  }
}

void orc_read_flags(void* h, unsigned char* solid, int* owner) {
  Oracle* o = (Oracle*)h;
  for (long n = 0; n < o->N; ++n) {
    if (solid) solid[n] = o->solid[n];
    if (owner) owner[n] = o->owner[n];
  }
}

void orc_read_phi(void* h, int body, double* out) {
  Oracle* o = (Oracle*)h;
  std::memcpy(out, o->bodies[body].phi.data(), sizeof(double) * o->N);
}

// Post-collision populations in the oracle's own velocity order, [q][cell].
void orc_read_populations(void* h, double* out) {
  Oracle* o = (Oracle*)h;
  std::memcpy(out, o->f.data(), sizeof(double) * o->f.size());
}
void orc_write_populations(void* h, const double* in) {
  Oracle* o = (Oracle*)h;
  std::memcpy(o->f.data(), in, sizeof(double) * o->f.size());
}
void orc_velocity_set(void* h, int* c, double* w) {
  Oracle* o = (Oracle*)h;
  for (int i = 0; i < o->L.Q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = o->L.c[i][a];
    w[i] = o->L.w[i];
  }
}

// The binary16 rounding of the storage model, for its test against an independent implementation.
double orc_round_binary16(double h) { return round_binary16(h); }

// Per-body total force/torque of the last step, and the parts
// [momentum exchange F,T | SC adhesion F,T | repulsion F,T] (18 per body).
void orc_read_body_forces(void* h, double* F, double* T, double* parts) {
  Oracle* o = (Oracle*)h;
  for (size_t b = 0; b < o->bodies.size(); ++b) {
    for (int a = 0; a < 3; ++a) {
      if (F) F[3 * b + a] = o->bodies[b].F[a];
      if (T) T[3 * b + a] = o->bodies[b].T[a];
    }
    if (parts)
      for (int k = 0; k < 18; ++k) parts[18 * b + k] = o->bodies[b].parts[k];
  }
}

void orc_get_bodies(void* h, double* X, double* V, double* W, double* Qo, double* M, double* I) {
  Oracle* o = (Oracle*)h;
  for (size_t b = 0; b < o->bodies.size(); ++b) {
    const Body& B = o->bodies[b];
    for (int a = 0; a < 3; ++a) {
      if (X) X[3 * b + a] = B.X[a];
      if (V) V[3 * b + a] = B.V[a];
      if (W) W[3 * b + a] = B.W[a];
    }
    if (Qo)
      for (int a = 0; a < 4; ++a) Qo[4 * b + a] = B.Q[a];
    if (M) M[b] = B.M;
    if (I)
      for (int a = 0; a < 9; ++a) I[9 * b + a] = B.Ibody[a];
  }
}

// Velocities only (positions are owned by the phase field).
void orc_set_body_velocity(void* h, int body, const double* V, const double* W) {
  Oracle* o = (Oracle*)h;
  for (int a = 0; a < 3; ++a) {
    if (V) o->bodies[body].V[a] = V[a];
    if (W) o->bodies[body].W[a] = W[a];
  }
}

// Hold (1) or release (0) a body; a held body is at rest (Sec. 4.3.2: the particles are held while
// the liquid settles, t = 0 is the release).
void orc_set_body_fixed(void* h, int body, int fixed) {
  Body& b = ((Oracle*)h)->bodies[body];
  b.fixed = fixed ? 1 : 0;
  if (b.fixed)
    for (int a = 0; a < 3; ++a) b.V[a] = b.W[a] = 0.0;
}

// Apply the body integrator to one body with a given force and torque (integrator pin).
void orc_integrate_body(void* h, int body, const double* F, const double* T) {
  Oracle* o = (Oracle*)h;
  Body& b = o->bodies[body];
  for (int k = 0; k < 18; ++k) b.parts[k] = 0.0;
  for (int a = 0; a < 3; ++a) { b.parts[a] = F[a]; b.parts[3 + a] = T[a]; }
  integrate_body(*o, b);
}

// Total fluid mass sum_x sum_i f_i (state populations; solid cells hold zero).
// Neumaier-compensated so that the check is limited by the state, not by the summation.
double orc_total_mass(void* h) {
  Oracle* o = (Oracle*)h;
  double s = 0, c = 0;
  for (size_t k = 0; k < o->f.size(); ++k) {
    double v = o->f[k], t = s + v;
    c += std::fabs(s) >= std::fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  return s + c;
}

// Fluid momentum sum c_i f_i of the state, and the body momentum sum M_B V_B.
void orc_total_momentum(void* h, double* fluid, double* bodies) {
  Oracle* o = (Oracle*)h;
  const long N = o->N;
  for (int a = 0; a < 3; ++a) { fluid[a] = 0; bodies[a] = 0; }
  for (int i = 0; i < o->L.Q; ++i) {
    double s = 0, c = 0;
    for (long n = 0; n < N; ++n) {
      double v = o->f[(size_t)i * N + n], t = s + v;
      c += std::fabs(s) >= std::fabs(v) ? (s - t) + v : (v - t) + s;
      s = t;
    }
    for (int a = 0; a < 3; ++a) fluid[a] += o->L.c[i][a] * (s + c);
  }
  for (const Body& b : o->bodies)
    for (int a = 0; a < 3; ++a) bodies[a] += b.M * b.V[a];
}

// Advance only the phase fields of all bodies by one step with the current V, omega
// (advection, optional kinetics, clamp, flags): used by the phase-field pins.
void orc_phase_only(void* h, int kinetics_on) {
  Oracle* o = (Oracle*)h;
  for (Body& b : o->bodies)
    for (int a = 0; a < 3; ++a) b.Xprev[a] = b.X[a];
  advect(*o);
  if (kinetics_on) kinetics(*o);
  flags_and_refill(*o);
}

}  // extern "C"
