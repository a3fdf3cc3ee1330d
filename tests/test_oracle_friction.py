"""Pins of the oracle's Coulomb friction (Eq. 6) and rolling resistance (Eq. 7).

A sphere on a plane inclined by theta (the plane is a kinematic geometry):
- without rotation (inverse inertia 0) it sticks iff tan(theta) <= mu_t and
  otherwise slides with a = g (sin theta - mu_t cos theta)  [block on a slope];
- with rotation and no rolling resistance it rolls without slip with
  a = g sin theta / (1 + I/(m l^2)), l the contact arm (= 5/7 g sin theta);
- with rolling resistance mu_r the rolling torque is capped at mu_r r N, so it
  stays at rest iff tan(theta) <= mu_r r / l and otherwise
  a = g (sin theta - mu_r (r/l) cos theta) / (1 + I/(m l^2)).
These fix the Coulomb bound on the physical normal impulse, the tangential
direction (maximum dissipation, Sec. 2.2) and the sign and size of the
rolling-resistance torque.
"""
import math

import numpy as np
import pytest

from oracle import Oracle, OracleParams, Geom
from oracle.binding import PLANE

E, NU, RHO, G = 1e9, 0.15, 2600.0, 9.81
R0 = 5e-3


def estar_wall():
    return 1.0 / ((1 - NU ** 2) / E + (1 - NU ** 2) / E)


def incline(theta_deg, mu_t, mu_r, rotate=True, n_it=60, dt=1e-5):
    th = math.radians(theta_deg)
    Rm = (1, 0, 0, 0, math.cos(th), -math.sin(th), 0, math.sin(th), math.cos(th))
    n = np.array([0.0, -math.sin(th), math.cos(th)])
    m = RHO * 4 / 3 * math.pi * R0 ** 3
    k = estar_wall() * math.sqrt(2 * R0) / 3.0
    d0 = (m * G * math.cos(th) / k) ** (2 / 3)       # static overlap, start near rest
    x = ((R0 - d0) * n)[None, :]
    p = OracleParams(rho=RHO, E=E, nu=NU, mu_t=mu_t, mu_r=mu_r, dt=dt, n_it=n_it,
                     gravity=(0, 0, -G), delta_floor=1e-10, damp_steps=4.5)
    plane = Geom(PLANE, c=(0, 0, 0), R=Rm, E=E, nu=NU, mu_t=mu_t, mu_r=mu_r)
    inv_I = None if rotate else np.zeros(1)
    o = Oracle(p, x, np.array([R0]), geoms=[plane], inv_I=inv_I)
    downhill = -np.array([0.0, math.cos(th), math.sin(th)])
    return o, downhill, m, d0, th


def downhill_accel(o, downhill, settle=500, span=2000, dt=1e-5):
    o.step(settle)
    _, v0, _ = o.state()
    o.step(span)
    _, v1, _ = o.state()
    return float((v1[0] - v0[0]) @ downhill) / (span * dt), v1[0]


@pytest.mark.parametrize("theta", [20.0, 26.0])
def test_block_sticks_below_friction_angle(theta):
    o, dn, m, d0, th = incline(theta, mu_t=0.5, mu_r=0.0, rotate=False)
    a, v = downhill_accel(o, dn)
    assert math.tan(th) < 0.5
    assert abs(a) < 1e-4 * G
    f, _ = o.geom_force(0)
    assert np.allclose(f, [0, 0, -m * G], rtol=0, atol=1e-6 * m * G)


@pytest.mark.parametrize("theta,mu", [(35.0, 0.5), (30.0, 0.3)])
def test_block_slides_above_friction_angle(theta, mu):
    o, dn, m, d0, th = incline(theta, mu_t=mu, mu_r=0.0, rotate=False)
    a, v = downhill_accel(o, dn)
    a_ref = G * (math.sin(th) - mu * math.cos(th))
    assert abs(a / a_ref - 1) < 2e-3, (a, a_ref)
    # the friction force opposes the sliding velocity (maximum dissipation)
    _, lam, *_ = o.contacts()[1:]
    pt = lam[0, 1:4]
    assert float(pt @ dn) < 0


def test_sphere_rolls_without_slip():
    o, dn, m, d0, th = incline(20.0, mu_t=0.5, mu_r=0.0, rotate=True, n_it=120)
    a, v = downhill_accel(o, dn)
    l = R0 - d0 / 2
    a_ref = G * math.sin(th) / (1 + 0.4 * R0 ** 2 / l ** 2)
    assert abs(a / a_ref - 1) < 2e-3, (a, a_ref)


def test_rolling_resistance_decelerates():
    mu_r = 0.1
    o, dn, m, d0, th = incline(20.0, mu_t=0.5, mu_r=mu_r, rotate=True, n_it=120)
    a, v = downhill_accel(o, dn)
    l = R0 - d0 / 2
    a_ref = G * (math.sin(th) - mu_r * (R0 / l) * math.cos(th)) / (1 + 0.4 * R0 ** 2 / l ** 2)
    assert abs(a / a_ref - 1) < 3e-3, (a, a_ref)


def test_rolling_resistance_holds_below_its_angle():
    o, dn, m, d0, th = incline(4.0, mu_t=0.5, mu_r=0.1, rotate=True, n_it=120)
    a, v = downhill_accel(o, dn)
    assert math.tan(th) < 0.1
    assert abs(a) < 1e-3 * G


def resting_on_floor(mu_t, rotate, floor_v):
    m = RHO * 4 / 3 * math.pi * R0 ** 3
    k = estar_wall() * math.sqrt(2 * R0) / 3.0
    d0 = (m * G / k) ** (2 / 3)
    p = OracleParams(rho=RHO, E=E, nu=NU, mu_t=mu_t, mu_r=0.0, dt=1e-5, n_it=60,
                     gravity=(0, 0, -G), delta_floor=1e-10)
    floor = Geom(PLANE, c=(0, 0, 0), v=floor_v, E=E, nu=NU, mu_t=mu_t, mu_r=0.0)
    inv_I = None if rotate else np.zeros(1)
    return Oracle(p, np.array([[0.0, 0.0, R0 - d0]]), np.array([R0]), geoms=[floor], inv_I=inv_I)


def test_moving_floor_drags_sphere_at_mu_g():
    """A floor sliding at u under a non-rotating sphere: kinetic friction
    accelerates it at mu g until it moves with the floor (the geometry's
    velocity enters the tangential rows)."""
    u, mu = 0.05, 0.3
    o = resting_on_floor(mu, False, (u, 0.0, 0.0))
    o.step(200)
    _, v0, _ = o.state()
    o.step(500)
    _, v1, _ = o.state()
    a = (v1[0, 0] - v0[0, 0]) / (500 * 1e-5)
    assert abs(a / (mu * G) - 1) < 2e-3
    o.step(2000)
    _, v2, _ = o.state()
    assert abs(v2[0, 0] / u - 1) < 1e-4
    g = o.geom(0)
    assert g.c[0] == pytest.approx(2700 * 1e-5 * u, rel=1e-12)


def test_rising_floor_carries_sphere():
    """A floor moving up at w: the sphere ends up moving with it (normal row)."""
    w = 0.01
    o = resting_on_floor(0.3, True, (0.0, 0.0, w))
    o.step(3000)
    _, v, _ = o.state()
    assert abs(v[0, 2] / w - 1) < 1e-3
    assert abs(v[0, 0]) < 1e-9
