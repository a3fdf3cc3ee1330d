"""Load-driven plate (dem_apply_plate_load) on the GPU against closed forms and
the FP64 oracle (orc_set_load).

Tolerances as in test_gpu_parity.py: trajectories within 1e-4 of their largest
values (FP32 solve against FP64); the plate's state is FP64 on both sides.
Masses and forces are powers of two, so that the GPU's float copies of the
load and of 1/M are exact.
"""
import math

import numpy as np
import pytest

from dem_cases import box_geoms, compressed_cloud, make_gpu, make_oracle, params
from paper_2501_05300_gb300 import beds

pytestmark = pytest.mark.gpu

DOWN = (1.0, 0.0, 0.0, 0.0, -1.0, 0.0, 0.0, 0.0, -1.0)


def test_free_fall_under_load():
    h, M, F, vx = 1e-4, 2.0, -32.0, 0.25
    p = params(dt=h, n_it=5, gravity=(0.0, 0.0, 0.0))
    plate = beds.GeomSpec(beds.PLANE, (0.0, 0.0, 1.0), DOWN, v=(vx, 0.0, 0.0))
    g = make_gpu(np.array([[5.0, 5.0, -5.0]]), np.array([0.005], np.float32), p, [plate])
    g.apply_plate_load([0], M, (0.0, 0.0, F), dof=4)
    k = 50
    g.step(k)
    G = g.read_geom(0)
    hf = float(np.float32(h))   # the library's time step is FP32
    assert abs(G.v[2] - k * hf * F / M) < 1e-14
    assert abs(G.c[2] - (1.0 + hf * hf * F / M * k * (k + 1) / 2)) < 1e-13
    assert G.v[0] == vx and abs(G.c[0] - vx * hf * k) < 1e-13
    g.close()


def test_loaded_plate_on_a_sphere_static_limit():
    r, F, M = 5e-3, 2.0, 0.0625
    p = params(dt=1e-5, n_it=40, delta_floor=1e-10, damp_steps=100.0)
    floor = beds.GeomSpec(beds.PLANE, (0.0, 0.0, 0.0))
    plate = beds.GeomSpec(beds.PLANE, (0.0, 0.0, 2 * r), DOWN)
    g = make_gpu(np.array([[0.0, 0.0, r]]), np.array([r], np.float32), p, [floor, plate])
    g.apply_plate_load([1], M, (0.0, 0.0, -F), dof=4)
    g.step(6000)
    m = 2600.0 * 4 / 3 * math.pi * np.float32(r) ** 3
    f_floor = g.read_forces(0)[0]
    f_plate = g.read_forces(1)[0]
    assert abs(f_plate[2] / F - 1) < 1e-4
    assert abs(-f_floor[2] / (F + m * 9.81) - 1) < 1e-4
    estar = 1.0 / (2 * (1 - 0.15 ** 2) / 1e9)
    k = estar * math.sqrt(2 * r) / 3.0
    x, v, _ = g.read_state()
    assert abs((r - x[0, 2]) / ((F + m * 9.81) / k) ** (2 / 3) - 1) < 1e-3
    assert abs((x[0, 2] + r - g.read_geom(1).c[2]) / (F / k) ** (2 / 3) - 1) < 1e-3
    g.close()


def loaded_case(n=1500, seed=21, n_it=50, dof=4, F=(0.0, 0.0, -64.0), M=0.5):
    """A compressed cloud in a frictional box; a box plate resting on its top,
    pressed down by a load (vertical dynamics), pulled sideways by its motor."""
    x, r = compressed_cloud(n, seed=seed)
    lo, hi = x.min(0) - 0.004, x.max(0) + 0.004
    geoms = box_geoms(lo, hi)
    c = (lo + hi) / 2
    top = float((x[:, 2] + r).max())
    geoms.append(beds.GeomSpec(beds.BOX, (c[0], c[1], top + 0.0047), he=(0.02, 0.015, 0.0045),
                               v=(0.01, 0.0, 0.0), mu_t=0.5, mu_r=0.02))
    return x, r, geoms, params(n_it=n_it), len(geoms) - 1, dict(mass=M, force=F, dof=dof)


@pytest.mark.parametrize("lanes,dof", [(0, 4), (2, 4), (0, 7)])
def test_loaded_plate_tracks_oracle(lanes, dof):
    x, r, geoms, p, gi, load = loaded_case(dof=dof)
    g = make_gpu(x, r, p, geoms, lanes=lanes)
    o = make_oracle(x, r, p, geoms)
    g.apply_plate_load([gi], load["mass"], load["force"], load["dof"])
    o.set_load([gi], load["mass"], load["force"], load["dof"])
    x0 = x.copy()
    z0 = o.geom(gi).c[2]
    for k in range(4):
        g.step(25)
        o.step(25)
        xg, vg, wg = g.read_state()
        xo, vo, wo = o.state()
        assert np.abs(vg - vo).max() < 1e-4 * np.abs(vo).max(), k
        assert np.abs(xg - xo).max() < 1e-4 * np.abs(xo - x0).max(), k
        pg, po = g.read_geom(gi), o.geom(gi)
        assert abs(pg.v[2] - po.v[2]) < 1e-4 * max(abs(po.v[2]), 1e-3), (k, pg.v[2], po.v[2])
        assert abs(pg.c[2] - po.c[2]) < 1e-4 * max(abs(po.c[2] - z0), 1e-9), k
        fg, fo = g.read_forces(gi)[0], o.geom_force(gi)[0]
        assert np.abs(fg - fo).max() < 1e-4 * np.abs(fo).max(), k
    assert abs(o.geom(gi).c[2] - z0) > 0          # the plate moved under its load
    assert abs(o.geom_force(gi)[0][2]) > 0        # and carries it
    g.close()


def test_loaded_plate_deterministic_and_resort_invariant():
    x, r, geoms, p, gi, load = loaded_case(n=3001, seed=4)
    out = []
    for every in (5, 5, 1000):
        g = make_gpu(x, r, p, geoms, resort_every=every)
        g.apply_plate_load([gi], load["mass"], load["force"], load["dof"])
        g.step(40)
        out.append((g.read_state()[1], np.array(g.read_geom(gi).c[:]), g.read_forces(gi)[0]))
        g.close()
    for o in out[1:]:
        for a, b in zip(o, out[0]):
            assert np.array_equal(a, b)


def test_group_members_and_motor():
    # a plate and a grouser in one group: one velocity; the motor sets both
    x, r, geoms, p, gi, load = loaded_case(n=600, seed=3)
    c = geoms[gi].c
    geoms.append(beds.GeomSpec(beds.BOX, (c[0], c[1], c[2] - 0.006), he=(0.003, 0.015, 0.0015),
                               v=(0.01, 0.0, 0.0)))
    gj = len(geoms) - 1
    g = make_gpu(x, r, p, geoms)
    o = make_oracle(x, r, p, geoms)
    g.apply_plate_load([gi, gj], 0.5, (0.0, 0.0, -64.0), 4)
    o.set_load([gi, gj], 0.5, (0.0, 0.0, -64.0), 4)
    g.step(20)
    o.step(20)
    g.apply_plate_velocity(gj, (0.03, 0.0, 0.0))
    o.set_geom_velocity(gj, (0.03, 0.0, 0.0))
    g.step(20)
    o.step(20)
    a, b = g.read_geom(gi), g.read_geom(gj)
    assert a.v[0] == b.v[0] == 0.03 and a.v[2] == b.v[2]
    assert abs(a.v[2] - o.geom(gi).v[2]) < 1e-4 * max(abs(o.geom(gi).v[2]), 1e-3)
    g.close()


def test_checkpoint_restores_the_group():
    x, r, geoms, p, gi, load = loaded_case(n=600, seed=3)
    g = make_gpu(x, r, p, geoms)
    g.apply_plate_load([gi], load["mass"], load["force"], load["dof"])
    g.step(10)
    h = g.save_checkpoint()
    g.step(15)
    ref = (g.read_state()[1], np.array(g.read_geom(gi).c[:]), np.array(g.read_geom(gi).v[:]))
    g.restore_checkpoint(h)
    g.step(15)
    out = (g.read_state()[1], np.array(g.read_geom(gi).c[:]), np.array(g.read_geom(gi).v[:]))
    for a, b in zip(out, ref):
        assert np.array_equal(a, b)
    g.free_checkpoint(h)
    g.close()


def test_plate_load_errors():
    from paper_2501_05300_gb300.dem import DEM_ERR_ARG, DemError
    x, r, geoms, p, gi, load = loaded_case(n=200, seed=3)
    g = make_gpu(x, r, p, geoms)
    for bad in (dict(geoms=[gi], mass=0.0, force=(0, 0, -1), dof=4),
                dict(geoms=[gi], mass=1.0, force=(0, 0, -1), dof=0),
                dict(geoms=[gi], mass=1.0, force=(0, 0, -1), dof=9),
                dict(geoms=[99], mass=1.0, force=(0, 0, -1), dof=4),
                dict(geoms=[gi, gi], mass=1.0, force=(0, 0, -1), dof=4)):
        with pytest.raises(DemError) as e:
            g.apply_plate_load(**bad)
        assert e.value.status == DEM_ERR_ARG
    g.apply_plate_load([gi], 1.0, (0, 0, -1), 4)
    with pytest.raises(DemError):
        g.apply_plate_load([gi], 1.0, (0, 0, -1), 4)     # already in a group
    with pytest.raises(DemError):                          # no adjoint through a dynamic plate
        g.record(2, 1)
    g.close()


def test_load_ramp_tracks_oracle():
    # the normal load applied gradually (dem_set_plate_load between steps)
    x, r, geoms, p, gi, load = loaded_case(n=1500, seed=21)
    g = make_gpu(x, r, p, geoms)
    o = make_oracle(x, r, p, geoms)
    g.apply_plate_load([gi], load["mass"], (0.0, 0.0, 0.0), 4)
    o.set_load([gi], load["mass"], (0.0, 0.0, 0.0), 4)
    for k in range(40):
        F = (0.0, 0.0, -2.0 * (k + 1))      # exact in FP32
        g.set_plate_load(gi, F)
        o.set_load_force(gi, F)
        g.step(1)
        o.step(1)
    pg, po = g.read_geom(gi), o.geom(gi)
    assert abs(pg.v[2] - po.v[2]) < 1e-4 * max(abs(po.v[2]), 1e-3)
    _, vg, _ = g.read_state()
    _, vo, _ = o.state()
    assert np.abs(vg - vo).max() < 1e-4 * np.abs(vo).max()
    from paper_2501_05300_gb300.dem import DemError
    with pytest.raises(DemError):
        g.set_plate_load(0, (0.0, 0.0, -1.0))      # a wall: in no group
    g.close()
