"""Pins of the oracle's warm start (Sec. 2.2: the iterative solve starts from
the previous step's multipliers).

A system placed exactly in its static equilibrium, at rest, with every contact
warm-started at its static impulse, is a fixed point of the projected sweep:
the velocities v* + M^-1 G^T lambda are zero, each SPOOK row's residual
G v + Sigma lambda - b vanishes (the Hertz static limit lambda_n = dt k_n
delta^{3/2}), and every impulse lies inside its cone.  So one step with a single
sweep must return the static impulses unchanged.  From a cold start the same
sweep cannot: mass splitting and the coupling of tangential and rolling rows
through the sphere's rotation leave it far from static.  This fixes the key
matching (pairs and sphere-primitive contacts), the copy of normal and rolling
impulses and the projection of the world-frame tangential impulse onto the new
tangent basis.
"""
import math

import numpy as np

from oracle import Geom, Oracle, OracleParams
from oracle.binding import PLANE

E, NU, RHO, G, DT = 1e9, 0.15, 2600.0, 9.81, 1e-5
R0 = 5e-3
ESTAR = 1.0 / (2 * (1 - NU * NU) / E)


def kn(dstar):
    return ESTAR * math.sqrt(dstar) / 3.0


def mass():
    return RHO * 4 / 3 * math.pi * R0 ** 3


def static_column(n):
    """Spheres stacked on a floor at their static overlaps; warm-start keys and
    world-frame impulses (p_n, p_t, p_r) of every contact on its body a."""
    m = mass()
    z = [R0 - (n * m * G / kn(2 * R0)) ** (2 / 3)]
    for k in range(n - 1):
        d = ((n - 1 - k) * m * G / kn(R0)) ** (2 / 3)
        z.append(z[-1] + 2 * R0 - d)
    x = np.array([[0.0, 0.0, zz] for zz in z])
    keys, lam = [(0, -1)], [[n * m * G * DT, 0, 0, 0, 0, 0, 0]]
    for k in range(n - 1):
        keys.append((k, k + 1))                  # normal from b (upper) to a (lower): -z
        lam.append([(n - 1 - k) * m * G * DT, 0, 0, 0, 0, 0, 0])
    order = sorted(range(len(keys)), key=lambda i: keys[i])
    return x, [keys[i] for i in order], np.array([lam[i] for i in order])


def column_oracle(n, warm):
    p = OracleParams(rho=RHO, E=E, nu=NU, mu_t=0.5, mu_r=0.02, dt=DT, n_it=1,
                     gravity=(0, 0, -G), delta_floor=1e-10, damp_steps=4.5, eps_reg=0.0)
    x, keys, lam = static_column(n)
    floor = Geom(PLANE, c=(0, 0, 0), E=E, nu=NU, mu_t=0.5, mu_r=0.02)
    o = Oracle(p, x, np.full(n, R0), geoms=[floor])
    if warm:
        o.set_warmstart([k[0] for k in keys], [k[1] for k in keys], lam)
    return o, keys, lam


def test_warm_started_column_stays_static_after_one_sweep():
    n = 6
    o, keys, lam = column_oracle(n, warm=True)
    o.step(1)
    ka, kb, got, _, _ = o.contacts()
    assert list(zip(ka, kb)) == keys
    assert np.abs(got - lam).max() < 1e-9 * lam[:, 0].max()
    _, v, w = o.state()
    assert np.abs(v).max() < 1e-9 * G * DT and np.abs(w).max() == 0.0
    # the floor carries the whole column
    f, _ = o.geom_force(0)
    assert abs(-f[2] / (n * mass() * G) - 1) < 1e-9


def test_cold_started_column_is_not_static_after_one_sweep():
    n = 6
    o, keys, lam = column_oracle(n, warm=False)
    o.step(1)
    _, _, got, _, _ = o.contacts()
    assert np.abs(got[:, 0] - lam[:, 0]).max() > 1e-2 * lam[:, 0].max()
    _, v, _ = o.state()
    assert np.abs(v).max() > 1e-2 * G * DT


def incline_oracle(theta_deg, warm, mu_t=0.5, mu_r=0.2):
    """A sphere held on a plane inclined by theta by static friction and
    rolling resistance (both inside their cones: tan theta <= mu_t and
    l tan theta <= mu_r r), at its static overlap."""
    th = math.radians(theta_deg)
    Rm = (1, 0, 0, 0, math.cos(th), -math.sin(th), 0, math.sin(th), math.cos(th))
    nrm = np.array([0.0, -math.sin(th), math.cos(th)])
    up = np.array([0.0, math.cos(th), math.sin(th)])   # up the slope
    m = mass()
    d0 = (m * G * math.cos(th) / kn(2 * R0)) ** (2 / 3)
    x = ((R0 - d0) * nrm)[None, :]
    p = OracleParams(rho=RHO, E=E, nu=NU, mu_t=mu_t, mu_r=mu_r, dt=DT, n_it=1,
                     gravity=(0, 0, -G), delta_floor=1e-10, damp_steps=4.5, eps_reg=0.0)
    plane = Geom(PLANE, c=(0, 0, 0), R=Rm, E=E, nu=NU, mu_t=mu_t, mu_r=mu_r)
    o = Oracle(p, x, np.array([R0]), geoms=[plane])
    pn = m * G * math.cos(th) * DT
    pt = m * G * math.sin(th) * DT * up
    l = R0 - d0 / 2
    pr = l * np.cross(nrm, pt)              # cancels the friction torque -l n x p_t
    lam = np.concatenate([[pn], pt, pr])[None, :]
    assert np.linalg.norm(pt) <= mu_t * pn and np.linalg.norm(pr) <= mu_r * R0 * pn
    if warm:
        o.set_warmstart([0], [-1], lam)
    return o, lam


def test_warm_started_incline_keeps_friction_and_rolling_impulse():
    o, lam = incline_oracle(5.0, warm=True)
    o.step(1)
    _, _, got, _, _ = o.contacts()
    assert np.abs(got - lam).max() < 1e-9 * lam[0, 0]
    _, v, w = o.state()
    assert np.abs(v).max() < 1e-9 * G * DT and np.abs(w).max() < 1e-9
    o.step(5)                                 # and it stays there
    _, _, got, _, _ = o.contacts()
    assert np.abs(got - lam).max() < 1e-9 * lam[0, 0]


def test_cold_started_incline_spins_after_one_sweep():
    o, lam = incline_oracle(5.0, warm=False)
    o.step(1)
    _, _, got, _, _ = o.contacts()
    _, v, w = o.state()
    # the rolling row was updated with the old (zero) spin: friction torque unbalanced
    assert np.abs(got[0, 4:] - lam[0, 4:]).max() > 0.5 * np.abs(lam[0, 4:]).max()
    assert np.linalg.norm(got[0, 1:4] - lam[0, 1:4]) > 0.5 * np.linalg.norm(lam[0, 1:4])
    assert np.abs(w).max() > 1e-4
