"""GPU path (C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (FP32 GPU arithmetic vs FP64 oracle, same Jacobi schedule):
- contact sets (sphere-sphere and sphere-geometry): bit-exact;
- one step: impulses within 1e-5 of the largest impulse, contact by contact,
  and 1e-5 normwise; velocities within 1e-5 of the largest velocity;
- trajectories of up to 200 steps: velocities and displacements within 1e-4
  of their largest values.
Sizes span several thread blocks with a ragged tail (600, 3001 particles) and
two or more grid levels.
"""
import numpy as np
import pytest

from dem_cases import (box_geoms, canonical_gpu_contacts, compressed_cloud, make_gpu, make_oracle,
                       params)
from paper_2501_05300_gb300 import beds

pytestmark = pytest.mark.gpu


def contact_sets_equal(g, o):
    a, b, lam, dl = g.read_contacts()
    a, b, lam, order = canonical_gpu_contacts(a, b, lam)
    oa, ob, olam, odl, _ = o.contacts()
    ok = np.array_equal(a, oa) and np.array_equal(b, ob)
    return ok, (a, b, lam, dl[order]), (oa, ob, olam, odl)


def assert_impulses_close(lam, olam, tol):
    scale = np.abs(olam).max()
    assert scale > 0
    err = np.abs(lam - olam).max(axis=1) / scale
    assert err.max() < tol, (err.max(), np.argmax(err))
    assert np.linalg.norm(lam - olam) / np.linalg.norm(olam) < tol


def cloud_case(n, seed, n_it=60):
    x, r = compressed_cloud(n, seed=seed)
    lo, hi = x.min(0) - 0.004, x.max(0) + 0.004
    geoms = box_geoms(lo, hi)
    # a rotated box and a cylinder poking into the cloud
    c = (lo + hi) / 2
    th = 0.4
    Rm = (np.cos(th), -np.sin(th), 0.0, np.sin(th), np.cos(th), 0.0, 0.0, 0.0, 1.0)
    geoms.append(beds.GeomSpec(beds.BOX, (c[0], c[1], hi[2] - 0.002), Rm, (0.02, 0.01, 0.006),
                               mu_t=0.5, mu_r=0.02))
    geoms.append(beds.GeomSpec(beds.CYLINDER, (lo[0] + 0.01, lo[1] + 0.01, c[2]), he=(0.012, 0.0, 0.01),
                               mu_t=0.5, mu_r=0.02))
    return x, r, geoms, params(n_it=n_it)


@pytest.mark.parametrize("n,seed", [(600, 1), (3001, 2)])
def test_contact_set_bit_exact(n, seed):
    x, r, geoms, p = cloud_case(n, seed, n_it=1)
    g = make_gpu(x, r, p, geoms)
    o = make_oracle(x, r, p, geoms)
    g.step(1)
    o.step(1)
    ok, (a, b, lam, dl), (oa, ob, olam, odl) = contact_sets_equal(g, o)
    assert ok
    assert (b < 0).sum() > 20 and (b >= 0).sum() > n          # geometry and pairs both present
    assert len(np.unique(b[b < 0])) >= 4                        # several primitives hit
    assert np.allclose(dl, odl, rtol=1e-6, atol=1e-7 * np.abs(odl).max())
    g.close()


@pytest.mark.parametrize("n,seed,n_it", [(600, 3, 40), (3001, 4, 100)])
def test_one_step_impulses_and_velocities(n, seed, n_it):
    x, r, geoms, p = cloud_case(n, seed, n_it=n_it)
    rng = np.random.default_rng(seed)
    v = rng.uniform(-0.05, 0.05, (n, 3)).astype(np.float32)
    w = rng.uniform(-5, 5, (n, 3)).astype(np.float32)
    g = make_gpu(x, r, p, geoms, v=v, w=w)
    o = make_oracle(x, r, p, geoms, v=v, w=w)
    g.step(1)
    o.step(1)
    ok, (a, b, lam, dl), (oa, ob, olam, odl) = contact_sets_equal(g, o)
    assert ok
    assert_impulses_close(lam, olam, 1e-5)
    xg, vg, wg = g.read_state()
    xo, vo, wo = o.state()
    assert np.abs(vg - vo).max() < 1e-5 * np.abs(vo).max()
    assert np.abs(wg - wo).max() < 1e-5 * np.abs(wo).max()
    disp = np.abs(xo - x).max()
    assert np.abs(xg - xo).max() < 1e-5 * disp
    g.close()


def test_warm_started_steps_track_oracle():
    """20 steps with warm starts carried across two Morton re-sorts."""
    x, r, geoms, p = cloud_case(3001, 5, n_it=60)
    g = make_gpu(x, r, p, geoms, resort_every=7)
    o = make_oracle(x, r, p, geoms)
    for k in range(4):
        g.step(5)
        o.step(5)
        ok, (a, b, lam, dl), (oa, ob, olam, odl) = contact_sets_equal(g, o)
        assert ok, k
        assert_impulses_close(lam, olam, 1e-5)
    g.close()


def test_settling_trajectory_200_steps():
    """A lattice falling into an open box: 200 steps of dropping, impacts and
    friction; velocities and displacements within 1e-4."""
    b = beds.settling_box(500)
    p = params(n_it=100, dt=1e-4)
    x0 = b.x.copy()
    g = make_gpu(b.x, b.r, p, b.geoms)
    o = make_oracle(b.x, b.r, p, b.geoms)
    contacts = 0
    for k in range(4):
        g.step(50)
        o.step(50)
        contacts += len(o.contacts()[0])
        xg, vg, wg = g.read_state()
        xo, vo, wo = o.state()
        assert np.abs(vg - vo).max() < 1e-4 * np.abs(vo).max(), k
        assert np.abs(xg - xo).max() < 1e-4 * np.abs(xo - x0).max(), k
    assert contacts > 50
    fg, tg, _ = g.read_forces(0)
    fo, to = o.geom_force(0)
    assert np.abs(fg - fo).max() < 1e-4 * np.abs(fo).max()
    g.close()


@pytest.mark.parametrize("lanes", [0, 1, 2, 4, 8, 16])
def test_dense_trajectory_200_steps(lanes):
    """A compressed cloud in a box under gravity expands and collides for 200
    steps with warm starts; every sweep layout (two-pass, threads per particle,
    resident)."""
    x, r, geoms, p = cloud_case(1000, 12, n_it=50)
    x0 = x.copy()
    g = make_gpu(x, r, p, geoms, lanes=lanes)
    o = make_oracle(x, r, p, geoms)
    for k in range(4):
        g.step(50)
        o.step(50)
        xg, vg, wg = g.read_state()
        xo, vo, wo = o.state()
        assert np.abs(vg - vo).max() < 1e-4 * np.abs(vo).max(), k
        assert np.abs(wg - wo).max() < 1e-4 * np.abs(wo).max(), k
        assert np.abs(xg - xo).max() < 1e-4 * np.abs(xo - x0).max(), k
    g.close()


def test_pushed_plate_force_and_pose():
    """A cylinder plate driven into a compressed cloud at constant velocity:
    its force, torque and pose after 60 steps."""
    x, r, geoms, p = cloud_case(3001, 6, n_it=60)
    top = x[:, 2].max() + r.max()
    c = x.mean(0)
    geoms.append(beds.GeomSpec(beds.CYLINDER, (c[0], c[1], top + 0.0005), he=(0.02, 0.0, 0.002),
                               v=(0.0, 0.0, -0.02), mu_t=0.5, mu_r=0.02))
    gi = len(geoms) - 1
    g = make_gpu(x, r, p, geoms)
    o = make_oracle(x, r, p, geoms)
    g.step(60)
    o.step(60)
    fg, tg, sink = g.read_forces(gi)
    fo, to = o.geom_force(gi)
    assert abs(fo[2]) > 0
    assert np.abs(fg - fo).max() < 1e-4 * np.abs(fo).max()
    assert np.abs(tg - to).max() < 1e-4 * max(np.abs(to).max(), 1e-3 * np.abs(fo).max())
    pg = g.read_geom(gi)
    po = o.geom(gi)
    assert np.array(pg.c[:]) == pytest.approx(np.array(po.c), abs=1e-15)
    # sinkage: highest particle top under the plate at creation minus the plate bottom
    under = (x[:, 0] - c[0]) ** 2 + (x[:, 1] - c[1]) ** 2 <= 0.02 ** 2
    z_ref = (x[under, 2] + r[under].astype(np.float64)).max()
    assert sink == pytest.approx(z_ref - (po.c[2] - 0.002), abs=1e-12)
    g.close()


def test_momentum_conserved_without_walls():
    x, r = compressed_cloud(1200, seed=8)
    rng = np.random.default_rng(8)
    v = rng.uniform(-0.1, 0.1, (len(r), 3)).astype(np.float32)
    p = params(n_it=40, gravity=(0.0, 0.0, 0.0), mu_r=0.1)
    g = make_gpu(x, r, p, (), v=v)
    m = p["rho"] * 4 / 3 * np.pi * r.astype(np.float64) ** 3
    P0 = (m[:, None] * v).sum(0)
    g.step(30)
    _, vg, wg = g.read_state()
    P1 = (m[:, None] * vg).sum(0)
    # impulses are applied bit-identically at both ends; what remains is the
    # FP32 rounding of the velocity updates
    assert np.abs(P1 - P0).max() < 1e-5 * (m[:, None] * np.abs(vg)).sum()
    g.close()
