"""The periodic wraps of the CUDA library (csrc/periodic.h) on the CPU.

The helpers are compiled as plain C++ (the header needs no CUDA header) and checked against the
subtraction loops they replace: bit for bit wherever those loops end (|d| <= 2n), and for
arguments that would make such a loop run for ever (+-Inf, NaN, 1e300) they must return at once.
"""
import math
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1902_10432_gb300", "csrc")

SRC = r"""
#include <cstdio>
#include <cstdlib>
#include "periodic.h"
int main(int argc, char** argv) {
  // reads lines "kind n value" from stdin, prints the result's bits
  char kind[8];
  int n;
  unsigned long long bits;
  while (std::scanf("%7s %d %llx", kind, &n, &bits) == 3) {
    double v;
    static_assert(sizeof(v) == sizeof(bits), "");
    __builtin_memcpy(&v, &bits, 8);
    double r = kind[0] == 'm' ? cbl::mimg(v, n)
               : kind[0] == 'w' ? cbl::wrapd(v, n)
               : kind[0] == 'n' ? (double)cbl::wrapi_near((int)v, n) : (double)cbl::wrapi((int)v, n);
    __builtin_memcpy(&bits, &r, 8);
    std::printf("%016llx\n", bits);
  }
  return 0;
}
"""


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _val(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("periodic")
    src = d / "t.cpp"
    src.write_text(SRC)
    exe = d / "t"
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", HDR, str(src), "-o", str(exe)])

    def call(cases):
        inp = "".join("%s %d %016x\n" % (k, n, _bits(float(v))) for k, n, v in cases)
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, timeout=20, check=True).stdout
        return [_val(int(l, 16)) for l in out.split()]

    return call


def _mimg_loop(d, n):
    h = 0.5 * n
    while d >= h:
        d -= n
    while d < -h:
        d += n
    return d


def _wrap_loop(x, n):
    while x >= n:
        x -= n
    while x < 0:
        x += n
    return x


def test_bitwise_equal_to_the_loops_within_two_periods(run):
    rng = np.random.default_rng(5)
    cases, exp = [], []
    for n in (4, 7, 48, 100, 128, 256, 512):
        h = 0.5 * n
        vals = list(rng.uniform(-2 * n, 2 * n, 400)) + [h, -h, math.nextafter(h, 0), math.nextafter(-h, -1e9),
                                                         2.0 * n, -2.0 * n, 1.5 * n, -1.5 * n, n, -n, 0.0, -0.0,
                                                         math.nextafter(h, 0) - 1e-3]
        for v in vals:
            cases.append(("m", n, v))
            exp.append(_mimg_loop(v, n))
            cases.append(("w", n, v))
            exp.append(_wrap_loop(v, n))
    got = run(cases)
    for (k, n, v), g, e in zip(cases, got, exp):
        assert _bits(g) == _bits(e), (k, n, v, g, e)


def test_minimum_image_range(run):
    rng = np.random.default_rng(6)
    cases = [("m", 64, v) for v in rng.uniform(-1e6, 1e6, 200)]
    for (k, n, v), g in zip(cases, run(cases)):
        assert -n / 2 <= g < n / 2
        assert abs(math.remainder(v - g, n)) < 1e-6


def test_non_finite_and_huge_arguments_return(run):
    # the loops never end for these; the closed forms return NaN or a finite value in range
    cases = []
    for n in (4, 128):
        for v in (math.inf, -math.inf, math.nan, 1e300, -1e300, 2.0 ** 60, -(2.0 ** 60)):
            cases += [("m", n, v), ("w", n, v)]
    got = run(cases)
    for (k, n, v), g in zip(cases, got):
        if math.isfinite(v):
            lo, hi = (-n / 2, n / 2) if k == "m" else (0.0, n)
            assert math.isnan(g) or lo <= g <= hi, (k, n, v, g)
        else:
            assert math.isnan(g), (k, n, v, g)


def test_integer_wrap(run):
    cases = [("i", n, a) for n in (4, 5, 256) for a in range(-3 * n, 3 * n)]
    for (k, n, a), g in zip(cases, run(cases)):
        assert g == a % n


def test_division_free_wrap_over_its_range(run):
    # wrapi_near (tile coordinates) equals the modulo over [-2n, 3n)
    cases = [("n", n, a) for n in (4, 5, 37, 256) for a in range(-2 * n, 3 * n)]
    for (k, n, a), g in zip(cases, run(cases)):
        assert g == a % n
