"""The workloads at their full sizes, in the launch configurations the
benchmark uses, against the oracle (or, where the O(N^2) oracle cannot finish,
against the exact contact predicate on a sample).

- refined bed, 201,686 spheres squeezed to the settled contact density: one step
  against one oracle step (contact set bit-exact, impulses and velocities within
  1e-5), two-pass sweep, one kernel with 2 threads per particle, and the
  resident sweep (one cooperative kernel per step);
- triaxial cell, 50,000 spheres: one step against the oracle;
- fine bed, ~4 M spheres: every contact of 20,000 sampled particles against the
  exact FP64 predicate (KD-tree candidates, then the predicate on the double
  centres), one thread per particle (the autotuner's choice);
- batch of 36 refined beds, 5.48 M spheres: one step of the batch equals the
  same beds stepped one by one, bit for bit.
"""
import numpy as np
import pytest

from dem_cases import canonical_gpu_contacts, make_gpu, make_oracle, params
from paper_2501_05300_gb300 import beds, rules

pytestmark = pytest.mark.gpu


def squeezed(bed, s=0.885):
    c = bed.x.mean(0)
    return c + (bed.x - c) * s


def one_step_parity(x, r, geoms, p, lanes):
    g = make_gpu(x, r, p, geoms, lanes=lanes)
    o = make_oracle(x, r, p, geoms)
    g.step(1)
    o.step(1)
    a, b, lam, dl = g.read_contacts()
    a, b, lam, order = canonical_gpu_contacts(a, b, lam)
    oa, ob, olam, odl, _ = o.contacts()
    assert np.array_equal(a, oa) and np.array_equal(b, ob)
    scale = np.abs(olam).max()
    assert np.abs(lam - olam).max() < 1e-5 * scale
    _, vg, wg = g.read_state()
    _, vo, wo = o.state()
    assert np.abs(vg - vo).max() < 1e-5 * np.abs(vo).max()
    assert np.abs(wg - wo).max() < 1e-5 * np.abs(wo).max()
    g.close()
    return len(a)


@pytest.mark.parametrize("lanes", [0, 2, 16])
def test_refined_bed_full_size_one_step(lanes):
    bed = beds.refined_sinkage_bed()
    x = squeezed(bed)
    nit = rules.n_iterations(rules.network_length_refined(4.0, 5e-3, 40e-3, 2.0, 0.25, 0.14), 0.02)
    m = bed.material
    p = params(n_it=nit, rho=m.rho, mu_t=m.mu_t, mu_r=m.mu_r)
    nc = one_step_parity(x, bed.r, bed.geoms, p, lanes)
    assert bed.n == 201686 and nc > 2 * bed.n


def test_triaxial_cell_full_size_one_step():
    bed = beds.triaxial_cell(50_000, squeeze=0.095, v_top=-0.1)
    p = params(n_it=172, gravity=(0.0, 0.0, 0.0))
    nc = one_step_parity(bed.x, bed.r, bed.geoms, p, 2)
    assert nc > 2 * bed.n


def test_fine_bed_full_size_sampled_contacts():
    from scipy.spatial import cKDTree
    bed = beds.fine_shear_bed(1.82, 0.91)
    x = squeezed(bed)
    r = bed.r
    g = make_gpu(x, r, params(n_it=1), bed.geoms, lanes=1)
    g.step(1)
    a, b, lam, dl = g.read_contacts()
    g.close()
    n = bed.n
    assert n > 3_900_000
    ss = b >= 0
    lo, hi = np.minimum(a[ss], b[ss]).astype(np.int64), np.maximum(a[ss], b[ss]).astype(np.int64)
    got = np.unique(lo * n + hi)

    def found(keys):
        pos = np.searchsorted(got, keys)
        return (pos < len(got)) & (got[np.minimum(pos, len(got) - 1)] == keys)

    rng = np.random.default_rng(7)
    sample = rng.choice(n, 20_000, replace=False)
    tree = cKDTree(x)
    r64 = r.astype(np.float64)
    cand = tree.query_ball_point(x[sample], 2.0 * float(r.max()) * 1.001)
    checked = 0
    for i, js in zip(sample.tolist(), cand):
        js = np.array([j for j in js if j != i], dtype=np.int64)
        d = x[i] - x[js]
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        R = r64[i] + r64[js]
        keys = np.minimum(i, js) * n + np.maximum(i, js)
        touch = d2 < R * R
        assert found(keys[touch]).all(), i            # every true contact was found
        assert not found(keys[~touch]).any(), i       # and no false one
        checked += int(touch.sum())
    assert checked > 20_000


def test_batch_full_size_equals_one_by_one():
    specs = beds.batch_specs()
    kws = []
    for k, s in enumerate(specs):
        b = beds.batch_bed(s, seed=2505 + k)
        kws.append(dict(x=squeezed(b), r=b.r, geoms=b.geoms, n_it=s["n_it"]))
    from paper_2501_05300_gb300.dem import Batch, Bed
    shared = dict(rho=2600.0, mu_t=0.5, mu_r=0.02, dt=1e-5, delta_floor=1e-8, lanes=1)
    batch = Batch(kws, **shared)
    batch.step(2)
    _, vb, wb = batch.read_state()
    assert batch.n > 5_000_000
    for k in (0, 17, 35):
        kw = kws[k]
        one = Bed(kw["x"], kw["r"], geoms=kw["geoms"], n_it=kw["n_it"], **shared)
        one.step(2)
        _, v1, w1 = one.read_state()
        o = batch.offsets[k]
        assert np.array_equal(v1, vb[o:o + one.n]) and np.array_equal(w1, wb[o:o + one.n])
        one.close()
    batch.close()
