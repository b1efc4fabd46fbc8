"""The Bethe-lattice recursion of section 4.2 against the paper's printed critical point.

Pins: the printed rho_c and (Y_c, B_c, F_c) (tests/golden/bethe_critical.txt); (0, 0, 0) is a
fixed point at every density; the returned point is a fixed point with a singular Jacobian of
x - step(x) (where the branch ends); just below rho_c Newton's method finds no non-trivial fixed
point near it, just above it does.
"""
import os

import numpy as np
import pytest

from paper_1710_05155_gb300 import bethe


def _golden(golden_dir):
    out = {}
    for line in open(os.path.join(golden_dir, "bethe_critical.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_critical_point_matches_the_paper(golden_dir):
    g = _golden(golden_dir)
    rho, y, b, f = bethe.critical_density()
    # the paper prints five or six digits
    assert rho == pytest.approx(g["rho_c"], abs=2e-5)
    assert y == pytest.approx(g["Y_c"], abs=2e-5)
    assert b == pytest.approx(g["B_c"], abs=2e-6)
    assert f == pytest.approx(g["F_c"], abs=2e-5)


def test_fixed_point_structure():
    rho, y, b, f = bethe.critical_density()
    v = np.array([y, b, f])
    assert np.abs(bethe.step(v, rho) - v).max() < 1e-10
    assert abs(np.linalg.det(bethe.jacobian(v, rho) - np.eye(3))) < 1e-8
    for r in (0.3, 0.8, 0.9):
        assert (bethe.step(np.zeros(3), r) == 0).all()
    _, ok_above = bethe.fixed_point(rho + 1e-3, v)
    _, ok_below = bethe.fixed_point(rho - 1e-3, v)
    assert ok_above and not ok_below


def test_jacobian_matches_finite_differences():
    v, rho, h = np.array([0.6, 0.05, 0.4]), 0.85, 1e-7
    J = np.stack([(bethe.step(v + h * e, rho) - bethe.step(v - h * e, rho)) / (2 * h)
                  for e in np.eye(3)], axis=1)
    assert np.allclose(J, bethe.jacobian(v, rho), atol=1e-6)
