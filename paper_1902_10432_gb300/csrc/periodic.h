// Periodic wraps of lattice coordinates, shared by the host and device code of the library.
//
// Every helper has a fixed operation count: no loop whose trip count depends on the value, so a
// non-finite or huge argument yields a non-finite or meaningless result but the call always returns
// (a device thread never spins on a value that an unstable run produced). Within the range that the
// library's own callers produce (|argument| <= 2 n) each helper returns exactly what the plain
// subtraction loop would ("while (d >= n/2) d -= n; while (d < -n/2) d += n"): every subtraction of
// n moves the value towards zero, so it is exact in binary floating point.
//
// This header needs no CUDA header, so host-only tools and tests compile it as plain C++.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define CBL_HD __host__ __device__
#else
#define CBL_HD
#endif

namespace cbl {

// a mod n in [0, n) for integers (n > 0)
CBL_HD inline int wrapi(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// a mod n for a in [-2n, 3n), without a division (an integer division by a value known only at run
// time costs some twenty instructions): tile coordinates, whose origins lie within about half a
// lattice length outside [0, n) and whose offsets are below n, stay in that range. Equal to wrapi
// there.
CBL_HD inline int wrapi_near(int a, int n) {
  if (a < 0) a += n;
  if (a < 0) a += n;
  if (a >= n) a -= n;
  if (a >= n) a -= n;
  return a;
}

// Minimum image of a coordinate difference: the representative of d modulo n in [-n/2, n/2).
// |d| <= 2n: at most two exact shifts by n. Larger |d|: one closed-form reduction first.
// NaN stays NaN, +-Inf becomes NaN.
CBL_HD inline double mimg(double d, int n) {
  const double nn = (double)n, h = 0.5 * nn;
  if (fabs(d) > 2.0 * nn) d -= nn * rint(d / nn);
  if (d >= h) d -= nn;
  else if (d < -h) d += nn;
  if (d >= h) d -= nn;
  else if (d < -h) d += nn;
  return d;
}

// x modulo n in [0, n) (a body centre after a move): the same structure as mimg.
CBL_HD inline double wrapd(double x, int n) {
  const double nn = (double)n;
  if (fabs(x) > 2.0 * nn) x -= nn * floor(x / nn);
  if (x >= nn) x -= nn;
  else if (x < 0.0) x += nn;
  if (x >= nn) x -= nn;
  else if (x < 0.0) x += nn;
  return x;
}

}  // namespace cbl
