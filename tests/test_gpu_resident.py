"""Resident sweep layout (lanes = 16): all sweeps of a step in one cooperative
kernel, one block per SM.

It takes the two-pass layout's arithmetic (the same contact update, the same
shares summed in incidence order), so its trajectories equal the two-pass
layout's bit for bit; against the FP64 oracle it keeps the tolerances of the
other layouts (one step 1e-5, trajectories 1e-4 of the largest value).
Covered: geometry contacts, re-sorts, beds smaller than the grid (empty
blocks), beds whose incidence shares overflow shared memory (global spill),
and beds that cannot take the layout (load-driven groups: two-pass instead).
"""
import numpy as np
import pytest

from dem_cases import box_geoms, canonical_gpu_contacts, compressed_cloud, make_gpu, make_oracle, params
from test_gpu_parity import cloud_case

pytestmark = pytest.mark.gpu

RESIDENT = 16


def states(x, r, p, geoms, lanes, steps, **kw):
    g = make_gpu(x, r, p, geoms, lanes=lanes, **kw)
    g.step(steps)
    out = g.read_state()
    f = [g.read_forces(k)[0] for k in range(len(geoms))]
    info = g.info()
    g.close()
    return out, f, info


@pytest.mark.parametrize("n,seed,steps", [(3001, 2, 30), (40, 3, 10)])
def test_resident_equals_two_pass_bitwise(n, seed, steps):
    x, r, geoms, p = cloud_case(n, seed, n_it=40)
    (s0, f0, _), (s1, f1, info) = (states(x, r, p, geoms, lanes, steps, resort_every=7) for lanes in (0, RESIDENT))
    assert info.lanes == RESIDENT
    for a, b in zip(s0, s1):
        assert np.array_equal(a, b)
    for a, b in zip(f0, f1):
        assert np.array_equal(a, b)


def test_resident_one_step_matches_oracle():
    x, r, geoms, p = cloud_case(3001, 5, n_it=60)
    g = make_gpu(x, r, p, geoms, lanes=RESIDENT)
    o = make_oracle(x, r, p, geoms)
    g.step(1)
    o.step(1)
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


def test_resident_shares_spill_to_global_memory():
    # ~3,000 particles per block: their incidence shares do not fit in shared
    # memory and the rest go through the global share array
    n = 152 * 3000
    x, r = compressed_cloud(n, seed=44)
    lo, hi = x.min(0) - 0.004, x.max(0) + 0.004
    geoms = box_geoms(lo, hi)
    p = params(n_it=12)
    (s0, f0, _), (s1, f1, info) = (states(x, r, p, geoms, lanes, 3) for lanes in (0, RESIDENT))
    assert info.lanes == RESIDENT
    for a, b in zip(s0, s1):
        assert np.array_equal(a, b)
    for a, b in zip(f0, f1):
        assert np.array_equal(a, b)


def test_resident_deterministic():
    x, r, geoms, p = cloud_case(3001, 8, n_it=30)
    (s0, _, _), (s1, _, _) = (states(x, r, p, geoms, RESIDENT, 12) for _ in range(2))
    for a, b in zip(s0, s1):
        assert np.array_equal(a, b)


def test_resident_falls_back_with_load_driven_groups():
    from test_gpu_load import loaded_case
    x, r, geoms, p, gi, load = loaded_case(n=1500, seed=21)
    out = []
    for lanes in (0, RESIDENT):
        g = make_gpu(x, r, p, geoms, lanes=lanes)
        g.apply_plate_load([gi], load["mass"], load["force"], load["dof"])
        g.step(20)
        out.append((g.read_state()[1], np.array(g.read_geom(gi).c[:])))
        g.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
