"""Pins of the host-side rules (Eqs. 1, 8-10) against the paper's tables and
identities, and of the seeded bed generator."""
import math
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_2501_05300_gb300 import beds, rules

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def table3():
    rows = [l.split() for l in open(os.path.join(GOLD, "table3_uniform_beds.txt"))
            if l.strip() and not l.startswith("#")]
    return np.array(rows, dtype=float)


def test_timestep_rule_reproduces_table3():
    """Eq. 9 with rho = 2200 kg/m^3, sigma = 50 kPa and one tolerance eps gives
    Table 3's time steps within 10% (the table rounds to 2 digits)."""
    t = table3()
    d, dt = t[:, 0] * 1e-3, t[:, 3] * 1e-3
    # the simplified form dt = d sqrt(eps rho / (6 sigma)) of Sec. 2.2
    for eps in (0.0189,):
        pred = np.array([rules.timestep(di, eps, 2200.0, 50e3) for di in d])
        simple = d * np.sqrt(eps * 2200.0 / (6 * 50e3))
        assert np.allclose(pred, simple, rtol=1e-12)
        assert np.all(np.abs(pred / dt - 1) < 0.10), pred / dt


def test_iteration_rule_slope_matches_table3():
    """Eq. 8 with n_d = h/d (h = 600 mm) is linear in n_d with slope 0.1/eps;
    Table 3's N_it rise by that slope with eps = 0.02, up to a constant offset
    the paper does not state.  The table's N_it are multiples of 25, which over
    the n_d span of 50 leaves the fitted slope uncertain by about 7%."""
    t = table3()
    nd = 0.6 / (t[:, 0] * 1e-3)
    slope = np.polyfit(nd, t[:, 2], 1)[0]
    assert abs(slope / (0.1 / 0.02) - 1) < 0.08
    assert rules.n_iterations(50.0, 0.02) == 250
    assert rules.n_iterations(14.75, 0.02) == 74


def test_layer_identities():
    """z_n = eta d0 (r^{n+1}-1)/(r-1) and d_n = d0/r + (r-1)/(r eta) z_n (Sec. 2.1)."""
    for d0, r, eta in [(8.5e-3, 1.5, 2.0), (5e-3, 2.0, 4.0), (8.5e-3, 1.25, 10.0)]:
        zb = rules.layer_bottoms(d0, r, eta, 8)
        for n, z in enumerate(zb):
            assert abs(z - eta * d0 * (r ** (n + 1) - 1) / (r - 1)) < 1e-12
            dn = d0 / r + (r - 1) / (r * eta) * z
            assert abs(dn - d0 * r ** n) < 1e-12
        gam = rules.discrete_aggressiveness(r, eta)
        # the discrete profile is the continuous one with d_min = d0/r offset
        assert abs(rules.refinement_profile(zb[3], d0 / r, gam, 1.0) - d0 * r ** 3) < 1e-12


def test_refinement_profile_eq1():
    d = [rules.refinement_profile(z, 8.5e-3, 0.05, 30e-3) for z in (0.0, 0.1, 0.43, 0.5)]
    assert d[0] == pytest.approx(8.5e-3)
    assert d[1] == pytest.approx(8.5e-3 + 0.005)
    assert d[2] == pytest.approx(30e-3)          # z_max = 0.43
    assert d[3] == pytest.approx(30e-3)
    assert rules.z_max(8.5e-3, 0.05, 30e-3) == pytest.approx(0.43)


def test_network_length_eq10():
    # the refined sinkage bed: eta 4, d 5 -> 40 mm, r 2, z_max 0.14, h 0.25
    nd = rules.network_length_refined(4.0, 5e-3, 40e-3, 2.0, 0.25, 0.14)
    assert nd == pytest.approx(12 + 2.75)
    # a uniform bed has no refined layers: n_d = h / d
    assert rules.network_length_refined(4.0, 8.5e-3, 8.5e-3, 2.0, 0.6, 0.0) == pytest.approx(0.6 / 8.5e-3)


def test_refined_layers_follow_sec21():
    layers = beds.refined_layers()
    rs = [l[0] for l in layers][::-1]
    th = [l[1] for l in layers][::-1]
    assert rs == pytest.approx([2.5e-3, 5e-3, 10e-3, 20e-3])
    assert th[:3] == pytest.approx([0.02, 0.04, 0.08])     # thickness eta d_n, eta = 4
    assert sum(th) == pytest.approx(0.25)


@pytest.mark.parametrize("maker", [lambda: beds.refined_sinkage_bed(0.3, 0.3),
                                   lambda: beds.settling_box()])
def test_generated_beds_have_no_overlaps_and_paper_spread(maker):
    b = maker()
    x, r = b.x, b.r.astype(np.float64)
    tree = cKDTree(x)
    pairs = tree.query_pairs(2 * r.max(), output_type="ndarray")
    if len(pairs):
        d = np.linalg.norm(x[pairs[:, 0]] - x[pairs[:, 1]], axis=1)
        assert (d > r[pairs[:, 0]] + r[pairs[:, 1]]).all()
    # every sphere is inside the container
    assert (x[:, 0] - r >= 0).all() and (x[:, 1] - r >= 0).all() and (x[:, 2] - r >= 0).all()
    assert (x[:, 0] + r <= b.box[0]).all() and (x[:, 1] + r <= b.box[1]).all()


def test_refined_bed_radius_bands():
    b = beds.refined_sinkage_bed(0.3, 0.3)
    for rn in (2.5e-3, 5e-3, 10e-3, 20e-3):
        m = (b.r > 0.85 * rn) & (b.r < 1.15 * rn)
        assert m.sum() > 0
        assert b.r[m].min() >= 0.9 * rn * (1 - 1e-6) and b.r[m].max() <= 1.1 * rn * (1 + 1e-6)


def test_refined_bed_count_is_about_200k():
    b = beds.refined_sinkage_bed()
    assert 190_000 < b.n < 215_000


def test_radial_zones_follow_the_layer_rule():
    # the layer rule of Sec. 2.1 along a distance: d_n = growth d_{n-1},
    # shells eta d_n thick, the capped size filling the rest
    z = beds.radial_zones(5e-3, 1.5, 3.0, 20e-3, 0.35)
    for (lo, hi, d), nxt in zip(z, z[1:]):
        assert abs((hi - lo) - 3.0 * d) < 1e-12 and abs(nxt[0] - hi) < 1e-15
        assert abs(nxt[2] - min(1.5 * d, 20e-3)) < 1e-15
    assert z[-1][2] == 20e-3 and z[-1][1] == 0.35 and z[0] == (0.0, 0.015, 5e-3)


@pytest.mark.parametrize("mode", ["hemisphere", "cylinder"])
def test_radially_refined_bed_sizes_grow_with_distance_no_overlaps(mode):
    b = beds.radially_refined_bed(mode=mode)
    cx, cy, depth = 0.2, 0.2, 0.2
    dh = np.hypot(b.x[:, 0] - cx, b.x[:, 1] - cy)
    dist = np.hypot(dh, depth - b.x[:, 2]) if mode == "hemisphere" else dh
    zones = beds.radial_zones(5e-3, 1.5, 3.0, 20e-3, 1.0)
    for lo, hi, d in zones:
        inside = (dist >= lo) & (dist < hi)
        if inside.any():
            # every sphere of a zone has that zone's size (10% spread)
            assert (b.r[inside] >= 0.45 * d * 0.999).all() and (b.r[inside] <= 0.55 * d * 1.001).all()
    # sizes grow monotonically with the zone index
    assert np.corrcoef(dist, b.r)[0, 1] > 0.5
    tree = cKDTree(b.x)
    pairs = tree.query_pairs(2 * float(b.r.max()), output_type="ndarray")
    gap = np.linalg.norm(b.x[pairs[:, 0]] - b.x[pairs[:, 1]], axis=1) - (b.r[pairs[:, 0]] + b.r[pairs[:, 1]])
    assert gap.min() > 0


def table2():
    rows = [l.split() for l in open(os.path.join(GOLD, "table2_refined_beds.txt"))
            if l.strip() and not l.startswith("#")]
    return np.array(rows, dtype=float)


def test_shear_slice_counts_match_tables_2_and_3():
    # uniform slices (Table 3) at phi 0.636 in the 1.5 x 0.17 x 0.6 m container
    # (Sec. 3.3) hold the paper's counts; the three refined slices of the
    # shear protocol fall in Table 2's ranges for their d_max (5 % slack: the
    # table rounds to thousands)
    for d_mm, count, _, _ in table3():
        n = beds.shear_slice(d_min=d_mm * 1e-3).n
        assert abs(n / count - 1) < 0.06, (d_mm, n, count)
    for row in table2():
        d_max, g_lo, g_hi, c_lo, c_hi = row[1] * 1e-3, row[2], row[3], row[6], row[7]
        cfg = {15e-3: dict(growth=1.1, eta=4.0), 22.5e-3: dict(growth=1.25, eta=2.0),
               30e-3: dict(growth=2.0, eta=1.0)}[round(d_max, 4)]
        gamma = rules.discrete_aggressiveness(cfg["growth"], cfg["eta"])
        assert g_lo <= gamma <= g_hi
        n = beds.shear_slice(d_max=d_max, **cfg).n
        assert 0.95 * c_lo <= n <= 1.05 * c_hi, (d_max, n)


def test_shear_slice_plate_dimensions():
    # plate 300 mm long and 500 mm wide (wider than the 170 mm slice), grousers
    # 43 mm deep and 25.5 mm long at the bottom (Sec. 3.3)
    b = beds.shear_slice(d_max=30e-3, growth=2.0, eta=1.0)
    plate, grousers = b.geoms[b.plate], [b.geoms[g] for g in b.plate_parts[1:]]
    assert abs(2 * plate.he[0] - 0.3) < 1e-12 and abs(2 * plate.he[1] - 0.5) < 1e-12
    assert len(grousers) == 3
    for g in grousers:
        assert abs(2 * g.he[2] - 0.043) < 1e-12 and abs(2 * g.he[0] - 0.0255) < 1e-12
        # hanging from the plate's underside
        assert abs((g.c[2] + g.he[2]) - (plate.c[2] - plate.he[2])) < 1e-12
    assert b.box == (1.5, 0.17, 0.6)


def test_protocol_measures_and_errors():
    import bench
    t = np.linspace(0.001, 5.4, 5400)
    sink = np.where(t <= 2.5, 0.002 * t / 2.5, 0.002 + 0.01 * (t - 2.5) / 2.9)
    ft = np.where(t <= 2.5, 0.0, np.where(t <= 3.0, 2550 * 0.3 * np.sin(np.pi * (t - 2.5) / 0.5), 2550 * 0.25))
    m = bench.protocol_measures(t, sink, ft, 2.5, 3.0, 2550.0)
    assert abs(m["static_sinkage_m"] - 0.002) < 1e-5 and abs(m["dynamic_sinkage_m"] - 0.012) < 1e-12
    assert abs(m["peak_traction"] - 0.3) < 1e-4
    after = t > 2.5
    assert abs(m["avg_traction"] - float((ft[after] / 2550).mean())) < 1e-12
    ref = dict(static_sinkage_m=0.001, dynamic_sinkage_m=0.010, peak_traction=0.25, avg_traction=0.2)
    e, agg = bench.protocol_errors(m, ref, 0.043, 2550.0, 2550.0)
    assert abs(e["static_sinkage"] - (m["static_sinkage_m"] - 0.001) / 0.043) < 1e-15
    assert abs(e["peak_traction"] - (m["peak_traction"] - 0.25)) < 1e-15
    assert abs(agg - np.mean(np.abs(list(e.values())))) < 1e-15
