"""Long runs: the GPU and the FP64 oracle on the pressure-sinkage and
shear-displacement curves of a small refined bed.

Over thousands of steps the two trajectories separate (FP32 against FP64 in a
chaotic granular flow), so long runs are compared on the measured curves, with
the paper's normalised errors (Sec. 4, aggregate error): sinkage differences
over the grouser depth, force differences over the normal load.  The bar is a
mean normalised error of 2% over the run.

The bed is two layers (r = 5 mm under r = 2.5 mm, 10% spread) in a frictionless
bin, settled by the oracle with the generation friction of Sec. 3.1; both sides
then start from that state with cold warm starts.
"""
import numpy as np
import pytest

import oracle
from oracle import OracleParams
from paper_2501_05300_gb300 import beds

from dem_cases import make_gpu, make_oracle, oracle_geoms, params

pytestmark = pytest.mark.gpu

LX = LY = 0.08
STEPS, EVERY = 2000, 20


@pytest.fixture(scope="module")
def settled():
    x, r = beds.layered_bed(LX, LY, [(5e-3, 0.03), (2.5e-3, 0.015)], spread=0.1, seed=31)
    walls = beds.open_box_walls(LX, LY, 0.0)
    p = params(dt=2e-4, n_it=40, mu_t=0.1, mu_r=0.01)
    o = oracle.Oracle(OracleParams(**p), x, np.asarray(r, np.float32).astype(np.float64),
                      geoms=oracle_geoms(walls))
    o.step(1500)
    xs, vs, ws = o.state()
    assert np.percentile(np.abs(vs), 95) < 0.02     # at rest, give or take the rattlers
    return xs, r, walls, vs.astype(np.float32), ws.astype(np.float32)


def run_both(x, r, geoms, v, w, p, setup, sample):
    g = make_gpu(x, r, p, geoms, v=v, w=w)
    o = make_oracle(x, r, p, geoms, v=v, w=w)
    setup(g, o)
    out_g, out_o = [], []
    for _ in range(STEPS // EVERY):
        g.step(EVERY)
        o.step(EVERY)
        out_g.append(sample(g, True))
        out_o.append(sample(o, False))
    g.close()
    return np.array(out_g), np.array(out_o)


def surface_under(x, r, cx, cy, half):
    under = (np.abs(x[:, 0] - cx) <= half) & (np.abs(x[:, 1] - cy) <= half)
    return float((x[under, 2] + r[under]).max())


def test_pressure_sinkage_curve(settled):
    x, r, walls, v, w = settled
    cx = cy = LX / 2
    top = surface_under(x, r, cx, cy, 0.015)
    plate = beds.GeomSpec(beds.CYLINDER, (cx, cy, top + 0.002 - 1e-4), he=(0.015, 0.0, 0.002),
                          v=(0.0, 0.0, -0.05), mu_t=0.5, mu_r=0.02)
    geoms = list(walls) + [plate]
    gi = len(geoms) - 1
    p = params(dt=1e-5, n_it=60)

    def sample(s, gpu):
        f = s.read_forces(gi)[0] if gpu else s.geom_force(gi)[0]
        return f[2]

    fg, fo = run_both(x, r, geoms, v, w, p, lambda g, o: None, sample)
    scale = np.abs(fo).max()
    assert scale > 0.5            # the plate is pushing into the bed
    ne = np.mean(np.abs(fg - fo)) / scale
    print(f"pressure-sinkage: normalised force error {ne:.5f}, peak force {scale:.3f} N")
    assert ne < 0.02, ne


def test_shear_displacement_curve(settled):
    # grousered plate under a normal load (vertical dynamics), dragged along x
    x, r, walls, v, w = settled
    cx = cy = LX / 2
    h_grouser, t_plate = 0.004, 0.002
    top = surface_under(x, r, cx, cy, 0.015)
    zc = top + h_grouser + t_plate / 2 - 2e-4
    parts = [beds.GeomSpec(beds.BOX, (cx, cy, zc), he=(0.015, 0.015, t_plate / 2), mu_t=0.5, mu_r=0.02)]
    for gx in (-0.01, 0.0, 0.01):
        parts.append(beds.GeomSpec(beds.BOX, (cx + gx, cy, zc - t_plate / 2 - h_grouser / 2),
                                   he=(0.001, 0.015, h_grouser / 2), mu_t=0.5, mu_r=0.02))
    geoms = list(walls) + parts
    ids = list(range(len(walls), len(geoms)))
    F_N, M = 8.0, 0.25           # ~9 kPa on 0.03 x 0.03 m; exact in FP32
    p = params(dt=1e-5, n_it=60)

    def setup(g, o):
        g.apply_plate_load(ids, M, (0.0, 0.0, -F_N), 4)
        o.set_load(ids, M, (0.0, 0.0, -F_N), 4)
        for gid in ids:
            g.apply_plate_velocity(gid, (0.05, 0.0, 0.0))
            o.set_geom_velocity(gid, (0.05, 0.0, 0.0))

    def sample(s, gpu):
        fx = sum((s.read_forces(k)[0] if gpu else s.geom_force(k)[0])[0] for k in ids)
        z = s.read_geom(ids[0]).c[2] if gpu else s.geom(ids[0]).c[2]
        return fx, z

    sg, so = run_both(x, r, geoms, v, w, p, setup, sample)
    assert np.abs(so[:, 0]).max() > 0.05 * F_N           # traction builds up
    assert so[0, 1] - so[-1, 1] > 0                       # the loaded plate sinks
    ne_t = np.mean(np.abs(sg[:, 0] - so[:, 0])) / F_N
    ne_z = np.mean(np.abs(sg[:, 1] - so[:, 1])) / h_grouser
    print(f"shear-displacement: normalised traction error {ne_t:.5f}, sinkage error {ne_z:.5f}, "
          f"peak traction {np.abs(so[:, 0]).max():.3f} N, sinkage {so[0, 1] - so[-1, 1]:.2e} m")
    assert ne_t < 0.02, ne_t
    assert ne_z < 0.02, ne_z
