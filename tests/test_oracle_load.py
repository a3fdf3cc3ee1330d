"""Pins of the oracle's load-driven rigid groups (orc_set_load): a plate whose
vertical motion is an unknown of the solve, driven by a constant load.

Each is checked against something other than the oracle: the discrete free-fall
sum of the symplectic step, the Hertz static overlaps of a loaded stack, and the
impulse-momentum balance of particles plus plate.
"""
import math

import numpy as np
import pytest

from oracle import Geom, Oracle, OracleParams
from oracle.binding import PLANE

E, NU = 1e9, 0.15
DOWN = (1, 0, 0, 0, -1, 0, 0, 0, -1)   # local z (the plane's normal) = -z


def kn(dstar, E1=E, nu1=NU, E2=E, nu2=NU):
    estar = 1.0 / ((1 - nu1 ** 2) / E1 + (1 - nu2 ** 2) / E2)
    return estar * math.sqrt(dstar) / 3.0


def test_loaded_plate_free_fall_is_the_discrete_sum():
    # no contact: v_k = k h F/M, z_k = z_0 + h^2 F/M k(k+1)/2; x keeps its motor speed
    h, M, F, vx = 1e-4, 2.0, -30.0, 0.3
    p = OracleParams(dt=h, n_it=5, gravity=(0.0, 0.0, 0.0))
    plate = Geom(PLANE, c=(0.0, 0.0, 1.0), R=DOWN, v=(vx, 0.0, 0.0))
    o = Oracle(p, np.array([[5.0, 5.0, -5.0]]), np.array([0.005]), geoms=[plate])
    o.set_load([0], M, (0.0, 0.0, F), dof=4)
    k = 50
    o.step(k)
    g = o.geom(0)
    assert abs(g.v[2] - k * h * F / M) < 1e-12
    assert abs(g.c[2] - (1.0 + h * h * F / M * k * (k + 1) / 2)) < 1e-12
    assert g.v[0] == vx and abs(g.c[0] - vx * h * k) < 1e-12


def test_loaded_plate_on_a_sphere_static_limit():
    # floor | sphere | plate under load F: the plate carries F, the floor F + m g,
    # and the overlaps are the Hertz static ones (F / k_n)^{2/3}
    r, rho, g0, F, M = 5e-3, 2600.0, 9.81, 2.0, 0.05
    p = OracleParams(rho=rho, E=E, nu=NU, dt=1e-5, n_it=40, gravity=(0, 0, -g0),
                     delta_floor=1e-10, damp_steps=100.0)
    floor = Geom(PLANE, c=(0, 0, 0), E=E, nu=NU)
    plate = Geom(PLANE, c=(0, 0, 2 * r), R=DOWN, E=E, nu=NU)
    o = Oracle(p, np.array([[0.0, 0.0, r]]), np.array([r]), geoms=[floor, plate])
    o.set_load([1], M, (0.0, 0.0, -F), dof=4)
    o.step(6000)
    m = rho * 4 / 3 * math.pi * r ** 3
    f_floor, _ = o.geom_force(0)
    f_plate, _ = o.geom_force(1)
    assert abs(f_plate[2] / F - 1) < 1e-6          # the sphere pushes the plate up with F
    assert abs(-f_floor[2] / (F + m * g0) - 1) < 1e-6
    k = kn(2 * r)
    d_pl = (F / k) ** (2 / 3)
    d_fl = ((F + m * g0) / k) ** (2 / 3)
    x, v, _ = o.state()
    assert abs((r - x[0, 2]) / d_fl - 1) < 1e-4
    zp = o.geom(1).c[2]
    assert abs((x[0, 2] + r - zp) / d_pl - 1) < 1e-4
    assert abs(o.geom(1).v[2]) < 1e-7 and np.abs(v).max() < 1e-7


def _cloud(n=30, seed=3):
    rng = np.random.default_rng(seed)
    x = np.zeros((n, 3))
    k = 0
    while k < n:
        q = rng.uniform(-0.02, 0.02, 3) * (1, 1, 0.4) + (0, 0, 0.0135)
        if k == 0 or np.min(np.linalg.norm(x[:k] - q, axis=1)) > 0.011:
            x[k] = q
            k += 1
    v = rng.uniform(-0.2, 0.2, (n, 3))
    v[:, 2] -= 0.5                        # towards the plate below
    return x, np.full(n, 5e-3), v


def _momentum(o, M, r, rho):
    x, v, _ = o.state()
    m = rho * 4 / 3 * math.pi * r ** 3
    return (m[:, None] * v).sum(0) + M * np.array(o.geom(0).v)


def test_group_momentum_balance():
    # a fully dynamic plate (all three axes) below a cloud, no gravity: particle
    # plus plate momentum changes by exactly F t (zero without a load)
    rho, M = 2600.0, 0.3
    x, r, v = _cloud()
    for F in ((0.0, 0.0, 0.0), (0.4, -0.2, 1.5)):
        p = OracleParams(rho=rho, dt=1e-5, n_it=30, gravity=(0, 0, 0), mu_t=0.5, mu_r=0.05)
        plate = Geom(PLANE, c=(0, 0, 0.0), mu_t=0.4, mu_r=0.02)
        o = Oracle(p, x, r, v, geoms=[plate])
        o.set_load([0], M, F, dof=7)
        p0 = _momentum(o, M, r, rho)
        steps = 400
        o.step(steps)
        p1 = _momentum(o, M, r, rho)
        assert np.abs(np.array(o.geom(0).v) - np.array(F) * 1e-5 * steps / M).max() > 1e-3   # pushed
        expect = p0 + np.array(F) * 1e-5 * steps
        assert np.allclose(p1, expect, rtol=0, atol=1e-12 * max(1.0, np.abs(p0).max()))


def test_group_moves_with_its_members():
    # two primitives in one group move together; the prescribed axes stay prescribed
    p = OracleParams(dt=1e-4, n_it=5, gravity=(0, 0, 0))
    a = Geom(PLANE, c=(0.0, 0.0, 1.0), R=DOWN, v=(0.1, 0.0, 0.0))
    b = Geom(PLANE, c=(0.0, 0.0, 2.0), R=DOWN, v=(0.7, 0.0, 0.0))
    o = Oracle(p, np.array([[5.0, 5.0, -5.0]]), np.array([0.005]), geoms=[a, b])
    o.set_load([0, 1], 1.0, (0.0, 0.0, -2.0), dof=4)
    o.step(10)
    ga, gb = o.geom(0), o.geom(1)
    assert ga.v == gb.v                              # one body
    assert abs(ga.c[2] - 1.0 - (gb.c[2] - 2.0)) < 1e-15
    assert ga.v[0] == 0.1                            # the first member's motor speed


def test_load_force_changed_between_steps_free_fall():
    # a group in free flight (no contacts, no gravity on it): v_k = sum_j dt F_j / M
    # and z_k = z_0 + dt sum_j v_j, whatever the force does from step to step
    h, M = 1e-4, 2.0
    p = OracleParams(dt=h, n_it=5, gravity=(0.0, 0.0, 0.0))
    plate = Geom(PLANE, c=(0.0, 0.0, 1.0), R=(1, 0, 0, 0, -1, 0, 0, 0, -1))
    o = Oracle(p, np.array([[5.0, 5.0, -5.0]]), np.array([0.005]), geoms=[plate])
    o.set_load([0], M, (0.0, 0.0, 0.0), 4)
    forces = [-(k + 1) * 3.0 for k in range(20)]
    v, z = 0.0, 1.0
    for F in forces:
        o.set_load_force(0, (0.0, 0.0, F))
        o.step(1)
        v += h * F / M
        z += h * v
    g = o.geom(0)
    assert abs(g.v[2] - v) < 1e-14 and abs(g.c[2] - z) < 1e-14
    with pytest.raises(ValueError):
        Oracle(p, np.array([[5.0, 5.0, -5.0]]), np.array([0.005]), geoms=[plate]).set_load_force(0, (0, 0, 1))
