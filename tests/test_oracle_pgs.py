"""Pins of the oracle's coloured projected Gauss-Seidel solver (solver = 1).

Gauss-Seidel and Jacobi are two iterations for the same complementarity
problem: where it has one solution (no friction, no rolling resistance; the
compliant rows make it strictly convex) both must reach it.  The static pins
of the Jacobi solver hold for PGS too, and the colouring obeys the bounds of a
greedy colouring of the contact conflict graph.
"""
import math

import numpy as np
import pytest

from oracle import Geom, Oracle, OracleParams
from oracle.binding import PLANE

from test_oracle_normal_law import E, NU, kn


def cloud(n=60, seed=5):
    rng = np.random.default_rng(seed)
    r = rng.uniform(4e-3, 6e-3, n)
    k = int(np.ceil(n ** (1 / 3)))
    idx = np.arange(n)
    x = np.stack([idx % k, (idx // k) % k, idx // (k * k)], 1) * 0.0095 + 0.006
    x = x + rng.uniform(-3e-4, 3e-4, x.shape)
    return x, r


def test_pgs_and_jacobi_reach_the_same_solution():
    x, r = cloud()
    floor = Geom(PLANE, c=(0, 0, 0), mu_t=0.0, mu_r=0.0)
    out = []
    for solver, n_it in ((0, 4000), (1, 1500)):
        p = OracleParams(mu_t=0.0, mu_r=0.0, n_it=n_it, solver=solver, gravity=(0, 0, -9.81))
        o = Oracle(p, x, r, geoms=[floor])
        o.step(1)
        ka, kb, lam, dl, nn = o.contacts()
        out.append((ka, kb, lam, o.state()[1]))
    (ka0, kb0, l0, v0), (ka1, kb1, l1, v1) = out
    assert np.array_equal(ka0, ka1) and np.array_equal(kb0, kb1) and len(ka0) > 30
    assert np.abs(l0 - l1).max() < 1e-6 * np.abs(l0).max()
    assert np.abs(v0 - v1).max() < 1e-6 * np.abs(v0).max()


def test_pgs_converges_faster_than_jacobi():
    # same problem, few iterations: Gauss-Seidel is closer to the solution
    x, r = cloud(seed=6)
    floor = Geom(PLANE, c=(0, 0, 0), mu_t=0.0, mu_r=0.0)

    def impulses(solver, n_it):
        p = OracleParams(mu_t=0.0, mu_r=0.0, n_it=n_it, solver=solver)
        o = Oracle(p, x, r, geoms=[floor])
        o.step(1)
        return o.contacts()[2]

    ref = impulses(1, 3000)
    err_j = np.abs(impulses(0, 20) - ref).max()
    err_g = np.abs(impulses(1, 20) - ref).max()
    assert err_g < 0.5 * err_j


def test_pgs_resting_column_static_limit():
    n, r, rho, g = 5, 5e-3, 2600.0, 9.81
    p = OracleParams(rho=rho, E=E, nu=NU, mu_t=0.5, mu_r=0.02, dt=1e-5, n_it=10, gravity=(0, 0, -g),
                     delta_floor=1e-10, damp_steps=100.0, solver=1)
    x = np.array([[0.0, 0.0, r + 2 * r * k] for k in range(n)])
    floor = Geom(PLANE, c=(0, 0, 0), E=E, nu=NU, mu_t=0.5, mu_r=0.02)
    o = Oracle(p, x, np.full(n, r), geoms=[floor])
    o.step(4000)
    m = rho * 4 / 3 * math.pi * r ** 3
    f, _ = o.geom_force(0)
    assert abs(-f[2] / (n * m * g) - 1) < 1e-6
    ka, kb, lam, dl, nn = o.contacts()
    ss = kb >= 0
    for j, d in enumerate(np.sort(dl[ss])[::-1]):
        assert abs(d / ((n - 1 - j) * m * g / kn(r)) ** (2 / 3) - 1) < 1e-4
    assert o.colours() == 2     # a chain: alternate colours


def test_pgs_colour_count_bounds():
    x, r = cloud(80, seed=9)
    floor = Geom(PLANE, c=(0, 0, 0))
    o = Oracle(OracleParams(n_it=2, solver=1), x, r, geoms=[floor])
    o.step(1)
    ka, kb, *_ = o.contacts()
    deg = np.bincount(np.concatenate([ka, kb[kb >= 0]]), minlength=len(r))
    # the contacts of one body form a clique; a greedy colouring needs at most
    # (largest conflict degree + 1) colours
    conflict = max(deg[a] - 1 + (deg[b] - 1 if b >= 0 else 0) for a, b in zip(ka, kb))
    assert deg.max() <= o.colours() <= conflict + 1


def test_pgs_rejects_load_driven_groups():
    plate = Geom(PLANE, c=(0, 0, 1.0), R=(1, 0, 0, 0, -1, 0, 0, 0, -1))
    o = Oracle(OracleParams(solver=1), np.array([[0.0, 0.0, 0.5]]), np.array([0.005]), geoms=[plate])
    o.set_load([0], 1.0, (0.0, 0.0, -1.0), 4)
    with pytest.raises(ValueError):
        o.step(1)
