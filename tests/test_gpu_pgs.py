"""Coloured projected Gauss-Seidel (solver = 1) on the GPU against the oracle's.

Both sides colour the contacts greedily in the order of the same priority
(a mix of the stable contact key), so they sweep in the same Gauss-Seidel
order; tolerances are those of the Jacobi parity tests (FP32 against FP64):
one step 1e-5 of the largest impulse and velocity, 40 steps 1e-4.
"""
import numpy as np
import pytest

from dem_cases import canonical_gpu_contacts, make_gpu, make_oracle
from test_gpu_parity import cloud_case

pytestmark = pytest.mark.gpu


def pgs_case(n=600, seed=1, n_it=30):
    x, r, geoms, p = cloud_case(n, seed, n_it=n_it)
    p = dict(p)
    p["solver"] = 1
    return x, r, geoms, p


def test_pgs_one_step_matches_oracle():
    x, r, geoms, p = pgs_case()
    g = make_gpu(x, r, p, geoms)
    o = make_oracle(x, r, p, geoms)
    g.step(1)
    o.step(1)
    assert g.info().colours == o.colours() > 1
    a, b, lam, dl = g.read_contacts()
    a, b, lam, _ = canonical_gpu_contacts(a, b, lam)
    oa, ob, olam, odl, _ = o.contacts()
    assert np.array_equal(a, oa) and np.array_equal(b, ob)
    assert np.abs(lam - olam).max() < 1e-5 * np.abs(olam).max()
    _, vg, wg = g.read_state()
    _, vo, wo = o.state()
    assert np.abs(vg - vo).max() < 1e-5 * np.abs(vo).max()
    assert np.abs(wg - wo).max() < 1e-5 * np.abs(wo).max()
    g.close()


def test_pgs_trajectory_tracks_oracle():
    x, r, geoms, p = pgs_case(n=1000, seed=12, n_it=20)
    g = make_gpu(x, r, p, geoms, resort_every=7)
    o = make_oracle(x, r, p, geoms)
    for k in range(2):
        g.step(20)
        o.step(20)
        xg, vg, wg = g.read_state()
        xo, vo, wo = o.state()
        assert np.abs(vg - vo).max() < 1e-4 * np.abs(vo).max(), k
        assert np.abs(xg - xo).max() < 1e-4 * np.abs(xo - x).max(), k
    g.close()


def test_pgs_deterministic():
    x, r, geoms, p = pgs_case(n=3001, seed=2)
    out = []
    for _ in range(2):
        g = make_gpu(x, r, p, geoms)
        g.step(5)
        out.append(g.read_state())
        g.close()
    for u, v in zip(*out):
        assert np.array_equal(u, v)


def test_pgs_converges_faster_than_jacobi():
    x, r, geoms, p = pgs_case(n=3001, seed=3)

    def velocities(solver, n_it):
        q = dict(p, solver=solver, n_it=n_it)
        g = make_gpu(x, r, q, geoms)
        g.step(1)
        v = g.read_state()[1]
        g.close()
        return v

    ref = velocities(1, 2000)
    err_j = np.abs(velocities(0, 20) - ref).max()
    err_g = np.abs(velocities(1, 20) - ref).max()
    assert err_g < 0.5 * err_j, (err_g, err_j)


def test_pgs_rejections():
    from paper_2501_05300_gb300.dem import DEM_ERR_ARG, DemError
    x, r, geoms, p = pgs_case(n=200, seed=4)
    g = make_gpu(x, r, p, geoms)
    with pytest.raises(DemError) as e:
        g.apply_plate_load([len(geoms) - 1], 1.0, (0, 0, -1), 4)
    assert e.value.status == DEM_ERR_ARG
    with pytest.raises(DemError):
        g.record(2, 1)
    g.close()
