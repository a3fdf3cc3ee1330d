"""Batched beds (dem_create_batch) and the autotuner.

Beds advanced together in one object must give bit-identical results to the
same beds advanced one by one: every sum runs in stable-id order and each bed
keeps its own grids, sweep count, primitives and warm starts."""
import numpy as np
import pytest

from dem_cases import box_geoms, compressed_cloud, params
from paper_2501_05300_gb300 import beds

pytestmark = pytest.mark.gpu


def bed_list():
    out = []
    for seed, n, nit in ((31, 700, 20), (32, 1500, 35), (33, 3001, 50)):
        x, r = compressed_cloud(n, seed=seed)
        lo, hi = x.min(0) - 0.004, x.max(0) + 0.004
        g = box_geoms(lo, hi)
        c = x.mean(0)
        g.append(beds.GeomSpec(beds.CYLINDER, (c[0], c[1], hi[2] + 0.001), he=(0.01, 0.0, 0.002),
                               v=(0.0, 0.0, -0.05), mu_t=0.5, mu_r=0.02))
        out.append(dict(x=x, r=r, geoms=g, n_it=nit))
    return out


@pytest.mark.parametrize("lanes", [0, 2])
def test_batch_equals_beds_one_by_one(lanes):
    from paper_2501_05300_gb300.dem import Batch, Bed
    specs = bed_list()
    p = params()
    p.pop("n_it")
    p["delta_floor"] = 1e-8
    single = [Bed(s["x"], s["r"], geoms=s["geoms"], n_it=s["n_it"], resort_every=7, lanes=lanes, **p)
              for s in specs]
    batch = Batch(specs, resort_every=7, lanes=lanes, **p)
    assert batch.info().n_beds == 3
    for _ in range(3):
        batch.step(5)
        for b in single:
            b.step(5)
    xb, vb, wb = batch.read_state()
    ab, bb, lb, db = batch.read_contacts()
    for k, b in enumerate(single):
        o, m = batch.offsets[k], len(specs[k]["r"])
        x, v, w = b.read_state()
        assert np.array_equal(xb[o:o + m], x) and np.array_equal(vb[o:o + m], v)
        assert np.array_equal(wb[o:o + m], w)
        g0, ng = batch.geom_offsets[k], len(specs[k]["geoms"])
        for g in range(ng):
            fs, ts, ss = b.read_forces(g)
            fb, tb, sb = batch.read_forces(g0 + g)
            assert np.array_equal(fs, fb) and np.array_equal(ts, tb) and ss == sb
        a, bk, lam, dl = b.read_contacts()
        sel = (ab >= o) & (ab < o + m)
        key_b = np.where(bb[sel] >= 0, bb[sel] - o, bb[sel] + g0)
        got = sorted(zip((ab[sel] - o).tolist(), key_b.tolist(), map(tuple, lb[sel].tolist())))
        ref = sorted(zip(a.tolist(), bk.tolist(), map(tuple, lam.tolist())))
        assert got == ref
    for b in single:
        b.close()
    batch.close()


def test_autotune_picks_a_valid_configuration():
    from paper_2501_05300_gb300.dem import Bed
    x, r = compressed_cloud(5000, seed=41)
    lo, hi = x.min(0) - 0.004, x.max(0) + 0.004
    b = Bed(x, r, geoms=box_geoms(lo, hi), **params(n_it=30))
    lanes, resort = b.autotune(3)
    assert lanes in (0, 1, 2, 4, 8) and resort in (5, 10, 20, 50)
    info = b.info()
    assert info.lanes == lanes and info.resort_every == resort
    b.step(3)
    b.sync()
    b.close()
