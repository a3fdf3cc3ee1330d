"""Batched beds (dem_create_batch) and the autotuner.

Beds advanced together in one object must give bit-identical results to the
same beds advanced one by one: every sum runs in stable-id order and each bed
keeps its own grids, sweep count, primitives and warm starts."""
import numpy as np
import pytest

from dem_cases import box_geoms, canonical_gpu_contacts, compressed_cloud, make_oracle, params
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
    cap0 = b.info().contact_capacity
    lanes, resort = b.autotune(3)
    assert lanes in (0, 1, 2, 4, 8) and resort in (5, 10, 20, 50)
    info = b.info()
    assert info.lanes == lanes and info.resort_every == resort
    # contact storage sized from the measured contacts (here smaller than 8 n)
    assert info.contacts <= info.contact_capacity <= 1.5 * info.contacts + 1024 + 0.5 * info.contacts
    assert info.contact_capacity < cap0
    b.step(3)
    b.sync()
    b.close()


def batch_bed_contacts(batch, k, specs):
    """Bed k's contacts of the batch's last step in the bed's own numbering,
    oriented like the oracle's (body a = lower stable id)."""
    ab, bb, lb, db = batch.read_contacts()
    o, m = batch.offsets[k], len(specs[k]["r"])
    g0 = batch.geom_offsets[k]
    sel = (ab >= o) & (ab < o + m)
    a = ab[sel] - o
    b = np.where(bb[sel] >= 0, bb[sel] - o, bb[sel] + g0)
    return canonical_gpu_contacts(a, b, lb[sel])[:3]


@pytest.mark.parametrize("lanes", [0, 2])
def test_batch_beds_track_their_oracles(lanes):
    """Every bed of a batch of three uneven beds (700 / 1500 / 3001 spheres,
    N_it 20 / 35 / 50, a plate sinking into each) against its own FP64 oracle
    run: contact sets bit-exact and impulses within 1e-5 after one step; after
    15 steps (warm starts carried across two re-sorts) contact sets bit-exact,
    velocities and displacements within 1e-4 and floor and plate forces within
    1e-4."""
    from paper_2501_05300_gb300.dem import Batch
    specs = bed_list()
    p = params()
    p.pop("n_it")
    batch = Batch(specs, resort_every=7, lanes=lanes, **p)
    orcs = [make_oracle(s["x"], s["r"], params(n_it=s["n_it"]), s["geoms"]) for s in specs]
    for steps in (1, 14):
        batch.step(steps)
        for o in orcs:
            o.step(steps)
        xb, vb, wb = batch.read_state()
        for k, (s, o) in enumerate(zip(specs, orcs)):
            a, b, lam = batch_bed_contacts(batch, k, specs)
            oa, ob, olam, _, _ = o.contacts()
            assert np.array_equal(a, oa) and np.array_equal(b, ob), (steps, k)
            off, m = batch.offsets[k], len(s["r"])
            xo, vo, wo = o.state()
            if steps == 1:
                scale = np.abs(olam).max()
                assert np.abs(lam - olam).max() < 1e-5 * scale, k
                assert np.abs(vb[off:off + m] - vo).max() < 1e-5 * np.abs(vo).max(), k
            else:
                assert np.abs(vb[off:off + m] - vo).max() < 1e-4 * np.abs(vo).max(), k
                assert np.abs(wb[off:off + m] - wo).max() < 1e-4 * np.abs(wo).max(), k
                disp = np.abs(xo - s["x"]).max()
                assert np.abs(xb[off:off + m] - xo).max() < 1e-4 * disp, k
                # the floor carries the bed; the plate may not have reached it yet
                # (then both forces are exactly zero)
                for gi in (0, len(s["geoms"]) - 1):
                    fb, _, _ = batch.read_forces(batch.geom_offsets[k] + gi)
                    fo, _ = o.geom_force(gi)
                    assert gi != 0 or abs(fo[2]) > 0
                    assert np.abs(fb - fo).max() <= 1e-4 * np.abs(fo).max(), (k, gi)
    batch.close()
