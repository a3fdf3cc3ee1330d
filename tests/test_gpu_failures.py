"""Failure detection and recovery on the GPU, without faulting the GPU.

- Contact storage that overflows (total capacity or one body's list) grows and
  the steps from the last committed one run again: the results equal those of
  a bed created with enough capacity, bit for bit, and the oracle's.
- A non-finite velocity given by the caller is reported as DEM_ERR_NONFINITE
  and latches the bed.
- The resident sweep's bounded waits, made to give up at once through the
  DEM_TEST_SPIN_LIMIT knob, end the kernel with DEM_ERR_TIMEOUT; the bed still
  answers and the context stays usable for the next bed.
"""
import math

import numpy as np
import pytest

from dem_cases import (box_geoms, canonical_gpu_contacts, compressed_cloud, make_gpu, make_oracle,
                       params)
from paper_2501_05300_gb300 import beds, dem

pytestmark = pytest.mark.gpu


def same_state(g1, g2):
    x1, v1, w1 = g1.read_state()
    x2, v2, w2 = g2.read_state()
    return np.array_equal(x1, x2) and np.array_equal(v1, v2) and np.array_equal(w1, w2)


def test_total_capacity_overflow_grows_and_replays():
    """A 2000-sphere compressed cloud with room for 100 contacts (it has
    ~5000): the first step overflows, the arrays grow and the ten steps
    enqueued at once are re-run; they equal a bed created with enough
    capacity."""
    x, r = compressed_cloud(2000, seed=4)
    lo, hi = x.min(0) - 0.004, x.max(0) + 0.004
    p = params(n_it=20)
    small = make_gpu(x, r, p, box_geoms(lo, hi), contact_capacity=100, resort_every=3)
    big = make_gpu(x, r, p, box_geoms(lo, hi), resort_every=3)
    cap0 = small.info().contact_capacity
    small.step(10)
    big.step(10)
    small.sync()
    info = small.info()
    assert info.steps == 10 and info.contact_capacity > cap0
    assert info.contacts > cap0
    assert same_state(small, big)
    a1, b1, l1, d1 = small.read_contacts()
    a2, b2, l2, d2 = big.read_contacts()
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2) and np.array_equal(l1, l2)
    small.step(5)                   # and it goes on at the grown capacity
    big.step(5)
    assert same_state(small, big)
    small.close()
    big.close()


def test_overflow_mid_run_after_resorts_matches_oracle():
    """A lattice falling into an open box: its sphere-sphere contacts pass a
    capacity of 5 around step 180, after many re-sorts (the warm starts of the
    last committed step carry over into the re-run).  The run equals one with
    enough capacity bit for bit and tracks the oracle over 200 steps."""
    b = beds.settling_box(1000)
    p = params(n_it=100, dt=1e-4)
    small = make_gpu(b.x, b.r, p, b.geoms, contact_capacity=5, resort_every=7)
    big = make_gpu(b.x, b.r, p, b.geoms, resort_every=7)
    o = make_oracle(b.x, b.r, p, b.geoms)
    cap0 = small.info().contact_capacity
    grew_at = None
    for k in range(20):
        small.step(10)
        big.step(10)
        o.step(10)
        small.sync()
        if grew_at is None and small.info().contact_capacity > cap0:
            grew_at = k
        assert same_state(small, big), k
    assert grew_at is not None and grew_at > 0            # the overflow came mid-run
    assert (o.contacts()[1] >= 0).sum() > cap0
    xg, vg, _ = small.read_state()
    xo, vo, _ = o.state()
    assert np.abs(vg - vo).max() < 1e-4 * np.abs(vo).max()
    assert np.abs(xg - xo).max() < 1e-4 * np.abs(xo - b.x).max()
    small.close()
    big.close()


def crowded_sphere(m=34, seed=9):
    """One sphere (r 9.9 mm) touched by m spheres of the same radius band
    (r 5 mm) on a shell around it, each overlapping it by 0.1 mm: it owns m
    contacts, more than the 32 a body's list holds at creation."""
    rng = np.random.default_rng(seed)
    k = np.arange(m) + 0.5
    th = np.arccos(1 - 2 * k / m)
    ph = math.pi * (1 + 5 ** 0.5) * k
    u = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    x = np.vstack([[0.0, 0.0, 0.0], (9.9e-3 + 5e-3 - 1e-4) * u]) + 0.05
    r = np.concatenate([[9.9e-3], np.full(m, 5e-3)]).astype(np.float32)
    v = rng.uniform(-0.01, 0.01, (m + 1, 3)).astype(np.float32)
    return x, r, v


def test_one_body_list_overflow_grows_and_matches_oracle():
    x, r, v = crowded_sphere()
    p = params(n_it=40, gravity=(0.0, 0.0, 0.0))
    g = make_gpu(x, r, p, (), v=v)
    o = make_oracle(x, r, p, (), v=v)
    g.step(1)
    o.step(1)
    a, b, lam, dl = g.read_contacts()
    a, b, lam, _ = canonical_gpu_contacts(a, b, lam)
    oa, ob, olam, odl, _ = o.contacts()
    assert np.array_equal(a, oa) and np.array_equal(b, ob)
    assert (oa == 0).sum() == 34
    assert np.abs(lam - olam).max() < 1e-5 * np.abs(olam).max()
    g.step(4)
    o.step(4)
    _, vg, wg = g.read_state()
    _, vo, wo = o.state()
    assert np.abs(vg - vo).max() < 1e-4 * np.abs(vo).max()
    g.close()


def test_nonfinite_velocity_is_reported_and_latched():
    x, r = compressed_cloud(600, seed=11)
    v = np.zeros((len(r), 3), np.float32)
    v[123, 1] = np.nan
    g = make_gpu(x, r, params(n_it=10), v=v)
    g.step(1)
    with pytest.raises(dem.DemError) as e:
        g.sync()
    assert e.value.status == dem.DEM_ERR_NONFINITE
    with pytest.raises(dem.DemError) as e:
        g.step(1)
    assert e.value.status == dem.DEM_ERR_STATE
    with pytest.raises(dem.DemError) as e:   # the bed answers, with its latched fault
        g.info()
    assert e.value.status == dem.DEM_ERR_NONFINITE
    g.close()


def test_resident_wait_timeout_is_reported_and_context_stays_usable(monkeypatch):
    x, r = compressed_cloud(3000, seed=12)
    lo, hi = x.min(0) - 0.004, x.max(0) + 0.004
    p = params(n_it=30)
    monkeypatch.setenv("DEM_TEST_SPIN_LIMIT", "1")
    g = make_gpu(x, r, p, box_geoms(lo, hi), lanes=16)
    monkeypatch.delenv("DEM_TEST_SPIN_LIMIT")
    g.step(2)
    with pytest.raises(dem.DemError) as e:
        g.sync()
    assert e.value.status == dem.DEM_ERR_TIMEOUT
    with pytest.raises(dem.DemError) as e:
        g.step(1)
    assert e.value.status == dem.DEM_ERR_STATE
    with pytest.raises(dem.DemError) as e:   # the bed answers, with its latched fault
        g.info()
    assert e.value.status == dem.DEM_ERR_TIMEOUT
    g.close()
    # a new bed on the same context steps and matches the two-pass layout
    g1 = make_gpu(x, r, p, box_geoms(lo, hi), lanes=16)
    g2 = make_gpu(x, r, p, box_geoms(lo, hi), lanes=0)
    g1.step(3)
    g2.step(3)
    assert same_state(g1, g2)
    g1.close()
    g2.close()
