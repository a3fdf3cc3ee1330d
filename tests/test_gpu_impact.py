"""Newton impact stage on the GPU against the FP64 oracle's.

Tolerances as for the other parity tests: one step 1e-5 of the largest value
(FP32 against FP64), trajectories 1e-4.  Impacting velocities are kept far from
the threshold, so both sides classify every contact alike and report the same
number of impacts.
"""
import numpy as np
import pytest

from dem_cases import box_geoms, compressed_cloud, make_gpu, make_oracle, params
from paper_2501_05300_gb300 import beds

pytestmark = pytest.mark.gpu

R = 5e-3
DELTA = 1e-9


def both(x, r, p, geoms=(), v=None, steps=1, **kw):
    g = make_gpu(x, r, p, geoms, v=v, **kw)
    o = make_oracle(x, r, p, geoms, v=v)
    g.step(steps)
    o.step(steps)
    return g, o


def test_head_on_pair_and_chain():
    p = params(mu_t=0.0, mu_r=0.0, n_it=400, gravity=(0.0, 0.0, 0.0), restitution=0.5, impact_speed=0.1)
    x = np.array([[0.0, 0.0, 0.0], [2 * R - DELTA, 0.0, 0.0], [4 * R - 2 * DELTA, 0.0, 0.0]])
    v = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    g, o = both(x, np.full(3, R), p, v=v)
    assert g.info().impacts == o.impacts() == 1
    vg, vo = g.read_state()[1], o.state()[1]
    assert np.abs(vg - vo).max() < 1e-5
    g.close()


def test_floor_rebound_and_floor_force():
    p = params(mu_t=0.0, mu_r=0.0, n_it=40, restitution=0.8, impact_speed=0.1)
    floor = beds.GeomSpec(beds.PLANE, (0.0, 0.0, 0.0), mu_t=0.0, mu_r=0.0)
    x = np.array([[0.0, 0.0, R - DELTA], [0.05, 0.0, R - DELTA]])
    v = np.array([[0.0, 0.0, -2.0], [0.0, 0.0, -0.01]])   # an impact and a resting contact
    g, o = both(x, np.full(2, R), p, [floor], v=v)
    assert g.info().impacts == o.impacts() == 1
    vg, vo = g.read_state()[1], o.state()[1]
    assert np.abs(vg - vo).max() < 1e-5 * 2.0
    fg, fo = g.read_forces(0)[0], o.geom_force(0)[0]
    assert abs(fg[2] / fo[2] - 1) < 1e-5
    g.close()


def impact_cloud(n, seed, speed=2.0):
    """A compressed cloud in a box, a third of the spheres thrown at speed."""
    x, r = compressed_cloud(n, seed=seed)
    lo, hi = x.min(0) - 0.004, x.max(0) + 0.004
    rng = np.random.default_rng(seed + 100)
    v = rng.normal(0.0, 0.002, (n, 3))
    fast = rng.random(n) < 1 / 3
    v[fast] = rng.normal(0.0, speed, (fast.sum(), 3))
    return x, r, box_geoms(lo, hi), v.astype(np.float32)


@pytest.mark.parametrize("e", [0.0, 0.6])
def test_cloud_one_step_matches_oracle(e):
    x, r, geoms, v = impact_cloud(1500, 7)
    p = params(n_it=60, restitution=e, impact_speed=0.3)
    g, o = both(x, r, p, geoms, v=v)
    assert g.info().impacts == o.impacts() > 50
    vg, vo = g.read_state()[1], o.state()[1]
    assert np.abs(vg - vo).max() < 1e-5 * np.abs(vo).max()
    for k in range(len(geoms)):
        fg, fo = g.read_forces(k)[0], o.geom_force(k)[0]
        assert np.abs(fg - fo).max() <= 1e-5 * np.abs(fo).max() + 1e-9
    g.close()


def test_cloud_trajectory_tracks_oracle():
    x, r, geoms, v = impact_cloud(1000, 9, speed=1.0)
    p = params(n_it=40, restitution=0.5, impact_speed=0.3)
    g = make_gpu(x, r, p, geoms, v=v)
    o = make_oracle(x, r, p, geoms, v=v)
    for k in range(3):
        g.step(10)
        o.step(10)
        xg, vg, _ = g.read_state()
        xo, vo, _ = o.state()
        assert np.abs(vg - vo).max() < 1e-4 * np.abs(vo).max(), k
        assert np.abs(xg - xo).max() < 1e-4 * np.abs(xo - x).max(), k
    g.close()


def test_no_impact_leaves_the_step_unchanged_bitwise():
    # the stage runs (threshold set) but no contact is fast enough; one step
    # only: the compressed cloud expands, and its later contacts do impact
    x, r, geoms, v = impact_cloud(1500, 3, speed=0.0)
    out = []
    for v_imp in (0.0, 0.3):
        g = make_gpu(x, r, params(n_it=30, restitution=0.5, impact_speed=v_imp), geoms, v=v)
        g.step(1)
        assert g.info().impacts == 0
        out.append(g.read_state())
        g.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_impacts_in_a_batch_equal_one_by_one():
    from paper_2501_05300_gb300.dem import Batch, Bed
    p = params(n_it=30, restitution=0.5, impact_speed=0.3)
    specs = []
    for k, (n, speed) in enumerate(((800, 2.0), (1200, 0.0), (600, 1.0))):
        x, r, geoms, v = impact_cloud(n, 20 + k, speed)
        specs.append(dict(x=x + 0.5 * k, r=r, geoms=[beds.GeomSpec(gg.type, tuple(np.add(gg.c, 0.5 * k)),
                                                                    tuple(gg.R), tuple(gg.he), mu_t=gg.mu_t,
                                                                    mu_r=gg.mu_r) for gg in geoms],
                          v=v, n_it=[30, 20, 40][k]))
    shared = {k: val for k, val in p.items() if k != "n_it"}
    batch = Batch(specs, **shared)
    batch.step(3)
    _, vb, _ = batch.read_state()
    for k, s in enumerate(specs):
        one = Bed(s["x"], s["r"], v=s["v"], geoms=s["geoms"], n_it=s["n_it"], **shared)
        one.step(3)
        o = batch.offsets[k]
        assert np.array_equal(one.read_state()[1], vb[o:o + one.n]), k
        one.close()
    batch.close()


def test_impact_arguments():
    from paper_2501_05300_gb300.dem import DemError
    x, r, geoms, v = impact_cloud(200, 4)
    with pytest.raises(DemError):
        make_gpu(x, r, params(restitution=1.5, impact_speed=0.3), geoms, v=v)
    g = make_gpu(x, r, params(restitution=0.5, impact_speed=0.3), geoms, v=v)
    with pytest.raises(DemError):
        g.record(2, 1)     # the adjoint does not reverse the impact stage
    g.close()


def test_impact_stage_with_gauss_seidel_matches_oracle():
    # the impact stage runs before either solver; with coloured Gauss-Seidel
    # after it the step still matches the oracle's
    x, r, geoms, v = impact_cloud(1200, 11)
    p = params(n_it=40, restitution=0.5, impact_speed=0.3, solver=1)
    g, o = both(x, r, p, geoms, v=v)
    assert g.info().impacts == o.impacts() > 30
    vg, vo = g.read_state()[1], o.state()[1]
    assert np.abs(vg - vo).max() < 1e-5 * np.abs(vo).max()
    g.close()


def test_impact_stage_enabled_between_steps():
    # dem_set_params turns the stage on (graphs rebuilt, buffers allocated):
    # the same trajectory as a bed created with it
    x, r, geoms, v = impact_cloud(800, 13)
    p_on = params(n_it=30, restitution=0.5, impact_speed=0.3)
    a = make_gpu(x, r, p_on, geoms, v=v)
    b = make_gpu(x, r, params(n_it=30), geoms, v=v)
    keys = ("dt", "n_it", "mu_t", "mu_r", "damp_steps", "e_H", "gravity", "kn_scale", "eps_reg")
    b.set_params(**{k: p_on[k] for k in keys}, restitution=0.5, impact_speed=0.3)
    a.step(5)
    b.step(5)
    assert a.info().impacts == b.info().impacts
    for u, w in zip(a.read_state(), b.read_state()):
        assert np.array_equal(u, w)
    b.set_params(**{k: p_on[k] for k in keys}, impact_speed=0.0)     # and off again
    b.step(2)
    assert b.info().impacts == 0
    a.close()
    b.close()
