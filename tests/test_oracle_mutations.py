"""The pins of the moving-wall term and of the MUSCL slope are sharp: a plausible mistake planted in
a copy of the oracle (on the CPU, in a temporary directory) makes them fail.

Each case copies oracle/ and the tests, replaces one expression of cbl_oracle.cpp, rebuilds the copy
and runs the pins that should catch the change; the run must fail. The wall term g of Sec. 3.2.2
(Eq. lb_bounce_back_us) is pinned by the Couette closed form and the one-step moving-body brute
force; the slope of the split MUSCL sweep (Sec. 3.3) by the one-sweep hand computation and the
second-order convergence test. (Where the link midpoint sits along c_i cannot matter: c_i . (omega x
c_i) = 0 and c_i x c_i = 0, so it drops out of both g and the torque.)
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WALL = "couette or moving_body"
SLOPE = "muscl"
CASES = {
    "wall term with factor 1": ("double g = 2.0 * r * L.w[i] * cu * 3.0;", "double g = 1.0 * r * L.w[i] * cu * 3.0;",
                                "test_oracle_lbm.py", WALL),
    "wall term with the wrong sign": ("double g = 2.0 * r * L.w[i] * cu * 3.0;",
                                      "double g = -2.0 * r * L.w[i] * cu * 3.0;", "test_oracle_lbm.py", WALL),
    "wall velocity omega x r reversed": ("cross(b.W, r, wr);", "cross(r, b.W, wr);", "test_oracle_lbm.py", WALL),
    "no (1 - |u|) factor, u > 0": ("face = p0 + 0.5 * (1.0 - uf) * mc_slope(p0 - pm1, p1 - p0);",
                                   "face = p0 + 0.5 * mc_slope(p0 - pm1, p1 - p0);", "test_oracle_phase.py", SLOPE),
    "no (1 - |u|) factor, u < 0": ("face = p1 - 0.5 * (1.0 + uf) * mc_slope(p1 - p0, p2 - p1);",
                                   "face = p1 - 0.5 * mc_slope(p1 - p0, p2 - p1);", "test_oracle_phase.py", SLOPE),
    "slope term doubled": ("face = p0 + 0.5 * (1.0 - uf) * mc_slope(p0 - pm1, p1 - p0);",
                           "face = p0 + (1.0 - uf) * mc_slope(p0 - pm1, p1 - p0);", "test_oracle_phase.py", SLOPE),
    "minmod instead of MC": ("std::min(std::min(2.0 * std::fabs(dm), 0.5 * std::fabs(dm + dp)), 2.0 * std::fabs(dp));",
                             "std::min(std::min(std::fabs(dm), 0.5 * std::fabs(dm + dp)), std::fabs(dp));",
                             "test_oracle_phase.py", SLOPE),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_planted_mistake_is_caught(name, tmp_path):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    old, new, test_file, expr = CASES[name]
    for d in ("oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("liboracle.so*", "__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    src = tmp_path / "oracle" / "cbl_oracle.cpp"
    text = src.read_text()
    assert text.count(old) == 1, name
    src.write_text(text.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join("tests", test_file), "-k", expr],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.stdout[-2000:], r.stderr[-2000:])
