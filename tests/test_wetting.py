"""Contact angle of the calibrated wetting parameter (Young's law, Sec. 2.1.1; wetting through
varrho_B, Sec. 3.2.3): at the varrho_B the table interpolates for a target angle, a sessile drop on
the FP64 oracle takes that angle within 2 degrees (a circle fitted to its mid-density contour)."""
import os
import sys

import pytest

from paper_1902_10432_gb300 import workloads

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_wetting_table as mw  # noqa: E402


@pytest.mark.parametrize("theta", [45.0, 90.0])
def test_interpolated_varrho_gives_the_target_angle(theta):
    v = workloads.varrho_for_angle(theta)
    measured, radius = mw.measure(v)
    print("target %.1f deg: varrho_B %.4f, measured %.2f deg (drop radius %.1f)" % (theta, v, measured, radius))
    assert abs(measured - theta) < 2.0
