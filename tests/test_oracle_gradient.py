"""Pins of the FP64 gradient oracle (oracle/torch_step.py).

The autograd gradient is only as good as the forward it differentiates, so the
forward is pinned to the C oracle (an independent implementation of the same
step), and the gradient to central finite differences of the C oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import OracleParams
from oracle import torch_step as ts
from paper_2501_05300_gb300 import beds

from dem_cases import oracle_geoms


def cell(n=64, squeeze=0.015, v_top=-0.05, mu_wall=0.0, seed=2505):
    b = beds.triaxial_cell(n, seed=seed, squeeze=squeeze, v_top=v_top)
    geoms = beds.cell_walls(*_bounds(b), v_top=v_top, mu_wall=mu_wall) if mu_wall else b.geoms
    return b.x, b.r.astype(np.float64), oracle_geoms(geoms)


def _bounds(b):
    lo = np.array([b.geoms[beds.WALL_XLO].c[0], b.geoms[beds.WALL_YLO].c[1], b.geoms[beds.FLOOR].c[2]])
    hi = np.array([b.geoms[beds.WALL_XHI].c[0], b.geoms[beds.WALL_YHI].c[1], b.geoms[beds.PLATEN].c[2]])
    return lo, hi


def weights(ng=6, seed=1):
    return np.random.default_rng(seed).normal(size=(ng, 3))


def oracle_objective(p, x, r, geoms, steps, W, v0=None):
    o = oracle.Oracle(p, x, r, v0, geoms=geoms)
    J = 0.0
    for _ in range(steps):
        o.step(1)
        J += sum(float(W[g] @ o.geom_force(g)[0]) for g in range(len(geoms)))
    return J, o


def moving(x, vmax=0.05, seed=5):
    return np.random.default_rng(seed).uniform(-vmax, vmax, x.shape)


@pytest.mark.parametrize("mu_wall,v_top,vmax,steps", [(0.0, -0.05, 0.0, 6), (0.3, -0.05, 0.0, 6),
                                                      (0.3, -1.0, 0.05, 12)])
def test_torch_forward_matches_c_oracle(mu_wall, v_top, vmax, steps):
    # the fast platen (10 um per step) moves contacts with it; the particles start moving
    x, r, geoms = cell(mu_wall=mu_wall, v_top=v_top)
    v0 = moving(x, vmax)
    p = OracleParams(n_it=30)
    W = weights()
    J, o = oracle_objective(p, x, r, geoms, steps, W, v0)
    xo, vo, wo = o.state()
    st = ts.TorchStepper(p, r, np.arange(len(r), dtype=np.int32), geoms)
    th = [torch.tensor(v, dtype=torch.float64) for v in (p.kn_scale, p.mu_t, p.mu_r)]
    Jt, xt, vt, wt = st.run(x, v0, np.zeros_like(x), th, steps, W)
    assert np.abs(xt.numpy() - xo).max() <= 1e-14
    assert np.abs(vt.numpy() - vo).max() <= 1e-10 * max(1.0, np.abs(vo).max())
    assert np.abs(wt.numpy() - wo).max() <= 1e-10 * max(1.0, np.abs(wo).max())
    assert abs(float(Jt) - J) <= 1e-10 * abs(J)
    assert abs(J) > 1.0   # the walls carry load


@pytest.mark.parametrize("mu_wall,v_top,vmax,steps", [(0.0, -0.05, 0.0, 5), (0.3, -0.05, 0.0, 8),
                                                      (0.3, -1.0, 0.05, 10)])
def test_autograd_gradient_matches_c_oracle_fd(mu_wall, v_top, vmax, steps):
    x, r, geoms = cell(n=200 if vmax else 64, mu_wall=mu_wall, v_top=v_top)
    v0 = moving(x, vmax)
    p = OracleParams(n_it=30)
    W = weights()
    th0 = np.array([p.kn_scale, p.mu_t, p.mu_r])
    J, g = ts.gradient(p, x, r, v0, np.zeros_like(x), geoms, th0, steps, W)
    fds = []
    for k, name in enumerate(("kn_scale", "mu_t", "mu_r")):
        h = 1e-5 * th0[k]
        vals = []
        for sgn in (1, -1):
            th = th0.copy()
            th[k] += sgn * h
            q = OracleParams(n_it=30, kn_scale=th[0], mu_t=th[1], mu_r=th[2])
            vals.append(oracle_objective(q, x, r, geoms, steps, W, v0)[0])
        fds.append((vals[0] - vals[1]) / (2 * h))
    # a stencil of +-1e-5 may still straddle a stick/slip switch of one contact:
    # 1e-4 of the component plus 1e-6 of the largest one
    fds = np.array(fds)
    assert np.all(np.abs(g - fds) <= 1e-4 * np.abs(fds) + 1e-6 * np.abs(fds).max()), (g, fds)
    if vmax:   # sliding and rolling contacts: every parameter matters
        assert np.all(np.abs(fds) > 1e-3 * np.abs(fds).max())


def test_gradient_zero_without_contacts():
    # spheres far from each other and from every wall: no force depends on theta
    x, r, _ = cell()
    x = x * 3.0
    geoms = oracle_geoms(beds.cell_walls(x.min(0) - 0.1, x.max(0) + 0.1, v_top=-0.05))
    p = OracleParams(n_it=10)
    J, g = ts.gradient(p, x, r, np.zeros_like(x), np.zeros_like(x), geoms, (1.0, 0.5, 0.02), 3, weights())
    assert J == 0.0 and np.all(g == 0.0)


def primitive_cloud(n=150, seed=7):
    from dem_cases import primitive_cloud as pc
    x, r, geoms = pc(n, seed)
    return x, r.astype(np.float64), oracle_geoms(geoms)


def _kinds(o, geoms):
    """Contact kinds of the box (index 5) and cylinder (6) in the last step:
    'face' when the normal is a local axis, else 'edge' (box) / 'rim' or
    'side' (cylinder)."""
    ka, kb, lam, dl, nn = o.contacts()
    kinds = set()
    for b, n in zip(kb, nn):
        g = -b - 1
        if g not in (5, 6):
            continue
        R = np.array(geoms[g].R).reshape(3, 3)
        nl = R.T @ n
        if g == 5:
            kinds.add("box face" if np.isclose(np.abs(nl).max(), 1.0, atol=1e-12) else "box edge/corner")
        else:
            axial = abs(nl[2])
            kinds.add("cyl cap" if np.isclose(axial, 1.0, atol=1e-12) else
                      ("cyl side" if axial < 1e-12 else "cyl rim"))
    return kinds


def test_torch_forward_matches_c_oracle_with_boxes_and_cylinders():
    x, r, geoms = primitive_cloud()
    v0 = moving(x, 0.05)
    p = OracleParams(n_it=30)
    W = weights(len(geoms))
    J, o = oracle_objective(p, x, r, geoms, 8, W, v0)
    kinds = _kinds(o, geoms)
    assert kinds == {"box face", "box edge/corner", "cyl cap", "cyl side", "cyl rim"}, kinds
    xo, vo, wo = o.state()
    st = ts.TorchStepper(p, r, np.arange(len(r), dtype=np.int32), geoms)
    th = [torch.tensor(v, dtype=torch.float64) for v in (p.kn_scale, p.mu_t, p.mu_r)]
    Jt, xt, vt, wt = st.run(x, v0, np.zeros_like(x), th, 8, W)
    assert np.abs(xt.numpy() - xo).max() <= 1e-14
    assert np.abs(vt.numpy() - vo).max() <= 1e-10 * max(1.0, np.abs(vo).max())
    assert np.abs(wt.numpy() - wo).max() <= 1e-10 * max(1.0, np.abs(wo).max())
    assert abs(float(Jt) - J) <= 1e-10 * abs(J)


def test_autograd_gradient_matches_c_oracle_fd_with_boxes_and_cylinders():
    x, r, geoms = primitive_cloud()
    v0 = moving(x, 0.05)
    p = OracleParams(n_it=30)
    W = np.zeros((len(geoms), 3))
    W[5] = (0.3, -0.2, 1.0)          # forces on the box and the cylinder
    W[6] = (-0.5, 0.4, 0.2)
    th0 = np.array([p.kn_scale, p.mu_t, p.mu_r])
    steps = 6
    J, g = ts.gradient(p, x, r, v0, np.zeros_like(x), geoms, th0, steps, W)
    fds = []
    for k in range(3):
        h = 1e-5 * th0[k]
        vals = []
        for sgn in (1, -1):
            th = th0.copy()
            th[k] += sgn * h
            q = OracleParams(n_it=30, kn_scale=th[0], mu_t=th[1], mu_r=th[2])
            vals.append(oracle_objective(q, x, r, geoms, steps, W, v0)[0])
        fds.append((vals[0] - vals[1]) / (2 * h))
    fds = np.array(fds)
    assert abs(J) > 0 and np.abs(fds).max() > 0
    assert np.all(np.abs(g - fds) <= 1e-4 * np.abs(fds) + 1e-6 * np.abs(fds).max()), (g, fds)
