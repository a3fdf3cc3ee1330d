"""Host logic of the calibration (no GPU): the Mohr-Coulomb fit of peak
triaxial states (Sec. 3.2) and the Gauss-Newton step.

- The fitted line is the common tangent of the Mohr circles: for states built
  from a known friction angle and cohesion, every circle (centre
  (sigma_1 + sigma_3) / 2, radius (sigma_1 - sigma_3) / 2) lies at distance
  equal to its radius from tau = c + sigma tan(phi), and the fit returns phi
  and c; with noise the fit equals numpy's least-squares line.
- Table 1's friction angles (golden fixture) are inside the range the fit
  reports for failure ratios built from them.
- A Gauss-Newton step on a linear residual lands on the least-squares
  solution (numpy.linalg.lstsq), and damping shortens it.
"""
import math
import os

import numpy as np
import pytest

from paper_2501_05300_gb300 import calibrate, triaxial

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1_triaxial.txt")


def table1():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    return np.array([float(r[4]) for r in rows])


def states(phi_deg, c, s3):
    """Peak sigma_1 of circles tangent to tau = c + sigma tan(phi), from the
    tangency condition itself: radius = centre sin(phi) + c cos(phi)."""
    phi = math.radians(phi_deg)
    s3 = np.asarray(s3, np.float64)
    # R = ((s1 + s3)/2) sin + c cos and R = (s1 - s3)/2  ->  solve for s1
    s1 = (s3 * (1 + math.sin(phi)) + 2 * c * math.cos(phi)) / (1 - math.sin(phi))
    return s1


@pytest.mark.parametrize("phi,c", [(34.3, 0.0), (30.0, 2e3), (40.0, 500.0)])
def test_fit_recovers_the_tangent_line(phi, c):
    s3 = np.array([5e3, 15e3, 25e3])
    s1 = states(phi, c, s3)
    ph, co = triaxial.mohr_coulomb_fit(s3, s1)
    assert ph == pytest.approx(phi, abs=1e-10)
    assert co == pytest.approx(c, abs=1e-7 * s1.max())
    # each circle touches the fitted line: distance from its centre = radius
    t = math.tan(math.radians(ph))
    for a, b in zip(s3, s1):
        centre, radius = 0.5 * (a + b), 0.5 * (b - a)
        dist = abs(co + t * centre) / math.sqrt(1 + t * t)
        assert dist == pytest.approx(radius, rel=1e-12)


def test_fit_equals_least_squares_line_with_noise():
    rng = np.random.default_rng(3)
    s3 = np.array([5e3, 15e3, 25e3])
    s1 = states(34.0, 0.0, s3) * (1 + rng.normal(0, 0.02, 3))
    ph, co = triaxial.mohr_coulomb_fit(s3, s1)
    K, b = np.polyfit(s3, s1, 1)
    assert math.sin(math.radians(ph)) == pytest.approx((K - 1) / (K + 1), rel=1e-12)
    assert co == pytest.approx(b / (2 * math.sqrt(K)), rel=1e-9, abs=1e-9)


def test_single_state_goes_through_origin_and_K_roundtrip():
    for phi in table1():
        K = triaxial.K_of_phi(phi)
        assert triaxial.phi_of_K(K) == pytest.approx(phi, abs=1e-12)
        ph, co = triaxial.mohr_coulomb_fit([10e3], [K * 10e3])
        assert ph == pytest.approx(phi, abs=1e-12) and co == 0.0
    # the paper's angles: 33.2 .. 34.9 deg, failure ratios 3.4 .. 3.7
    Ks = [triaxial.K_of_phi(p) for p in table1()]
    assert 3.4 < min(Ks) and max(Ks) < 3.7


def test_fit_rejects_non_frictional_data():
    with pytest.raises(ValueError):
        triaxial.mohr_coulomb_fit([5e3, 15e3], [4e3, 8e3])


def test_gauss_newton_step_solves_linear_least_squares():
    rng = np.random.default_rng(5)
    A = rng.normal(size=(3, 2))
    b = rng.normal(size=3)
    x0 = rng.normal(size=2)
    r0 = A @ x0 - b
    d = calibrate.gauss_newton_step(r0, A)
    x_ls, *_ = np.linalg.lstsq(A, b, rcond=None)
    assert np.allclose(x0 + d, x_ls, rtol=0, atol=1e-12)
    dd = calibrate.gauss_newton_step(r0, A, damping=1.0)
    assert np.linalg.norm(dd) < np.linalg.norm(d)
    # the damped step still decreases the residual
    assert np.linalg.norm(A @ (x0 + dd) - b) < np.linalg.norm(r0)
