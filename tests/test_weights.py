"""The FP32 lattice weights of the collision (csrc/weights.h) on the CPU.

The equilibria of Sec. 3.2.1 sum to rho because the weights sum to 1. The header is compiled as
plain C++ and its values are checked exactly, as rationals: each lies within 2 ulp of the exact
weight (1/3, 1/18, 1/36; 8/27, 2/27, 1/54, 1/216), each set sums to exactly 1 over its velocities,
and the FP32 values nearest to the weights do not (the mass that an FP32 collision using them would
add at every step).
"""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1902_10432_gb300", "csrc")

SRC = r"""
#include <cstdio>
#include "weights.h"
int main() {
  for (int i = 0; i < 19; ++i) std::printf("19 %d %a\n", i, (double)cbl::q19::wf_of(i));
  for (int i = 0; i < 27; ++i) std::printf("27 %d %a\n", i, (double)cbl::q27::wf_of(i));
  return 0;
}
"""

# exact weights by speed class, and the number of velocities in each class (Sec. 3.2.1)
EXACT = {
    19: [(Fraction(1, 3), 1), (Fraction(1, 18), 6), (Fraction(1, 36), 12)],
    27: [(Fraction(8, 27), 1), (Fraction(2, 27), 6), (Fraction(1, 54), 12), (Fraction(1, 216), 8)],
}


def _exact(q, i):
    k = 0
    for w, n in EXACT[q]:
        if i < k + n:
            return w
        k += n
    raise IndexError(i)


@pytest.fixture(scope="module")
def weights(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("weights")
    src = d / "t.cpp"
    src.write_text(SRC)
    exe = d / "t"
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-I", HDR, str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=20, check=True).stdout
    w = {19: [], 27: []}
    for line in out.split("\n"):
        if line:
            q, i, v = line.split()
            w[int(q)].append(float.fromhex(v))
    return w


def _ulp32(x):
    x = np.float32(x)
    return Fraction(float(np.nextafter(x, np.float32(np.inf)) - x))


@pytest.mark.parametrize("q", [19, 27])
def test_values_are_fp32_within_two_ulp(weights, q):
    assert len(weights[q]) == q
    for i, v in enumerate(weights[q]):
        assert float(np.float32(v)) == v  # an FP32 value
        assert abs(Fraction(v) - _exact(q, i)) <= 2 * _ulp32(v), (q, i, v)
    # one value per speed class, as the lattice's symmetry requires
    classes = {}
    for i, v in enumerate(weights[q]):
        classes.setdefault(_exact(q, i), set()).add(v)
    assert all(len(s) == 1 for s in classes.values())


@pytest.mark.parametrize("q", [19, 27])
def test_sum_is_exactly_one(weights, q):
    assert sum(Fraction(v) for v in weights[q]) == 1


@pytest.mark.parametrize("q,excess", [(19, Fraction(1, 2 ** 26)), (27, Fraction(1, 2 ** 27))])
def test_nearest_fp32_weights_do_not_sum_to_one(q, excess):
    # the reason for the set above: rounded to nearest, the weights sum to 1 + 1.49e-8 (D3Q19) or
    # 1 + 7.45e-9 (D3Q27)
    s = sum(Fraction(float(np.float32(float(w)))) * n for w, n in EXACT[q])
    assert s - 1 == excess


def test_fp32_equilibria_carry_no_mass_bias(weights):
    # The D3Q19 equilibria of 2e5 random cells evaluated in plain FP32 (every operation rounded,
    # Sec. 3.2.1's f_eq = w rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u)) and summed exactly: with the
    # nearest FP32 weights the sum exceeds rho by 1.6e-8 on average (the weights' 1.49e-8 plus the
    # rounding of the bracket), with the header's weights by the bracket's rounding alone (~1e-9).
    rng = np.random.default_rng(1)
    n = 200000
    f32 = np.float32
    rho = rng.uniform(0.1, 2.0, n).astype(f32)
    u = (0.05 * rng.standard_normal((n, 3))).astype(f32)
    uu = (u[:, 0] * u[:, 0] + u[:, 1] * u[:, 1] + u[:, 2] * u[:, 2]).astype(f32)
    c = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
         (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
         (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]

    def mean_excess(w):
        tot = np.zeros(n)
        for (cx, cy, cz), wi in zip(c, w):
            cu = (f32(cx) * u[:, 0] + f32(cy) * u[:, 1] + f32(cz) * u[:, 2]).astype(f32)
            f = (f32(wi) * rho * (f32(1) + f32(3) * cu + f32(4.5) * cu * cu - f32(1.5) * uu)).astype(f32)
            tot += f.astype(np.float64)
        return float(np.mean((tot - rho) / rho))

    nearest = [float(np.float32(float(_exact(19, i)))) for i in range(19)]
    assert mean_excess(nearest) > 1.4e-8
    assert abs(mean_excess(weights[19])) < 2e-9
