"""GPU adjoint (dem_record / dem_step_adjoint) against the FP64 gradient oracle
and against central finite differences of the GPU forward.

Tolerances.  The GPU step runs in FP32: one step's forces carry a relative
error of about 1e-6 (the per-step parity bar is 1e-5) and the adjoint sums
N_it * steps FP32 terms per contact, each with a relative rounding of 6e-8.
Gradients are compared component-wise against 2e-4 of the largest component
(the sum of a few thousand such roundings).  Central differences with
h = 1e-3 relative carry an O(h^2) truncation error and FP32 noise of about
1e-7 |J| / (2h theta); they are compared at 5e-3 of the largest component,
since a finite step may also cross a change of the active set (stick/slip,
opening contacts) that the derivative along the fixed active set does not see.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

from oracle import OracleParams
from oracle import torch_step as ts
from paper_2501_05300_gb300 import beds

from dem_cases import make_gpu, oracle_geoms, params, primitive_cloud

pytestmark = pytest.mark.gpu

THETA = (1.0, 0.5, 0.02)


def small_cell(n=200, n_it=30, mu_wall=0.0, resort_every=3, vmax=0.05, seed=11, **kw):
    """A pre-stressed triaxial cell whose particles start with random
    velocities (so that contacts slide and roll) and whose platen moves down
    at 0.5 m/s."""
    b = beds.triaxial_cell(n, squeeze=0.015, v_top=-0.5)
    geoms = b.geoms if not mu_wall else [replace(g, mu_t=mu_wall, mu_r=mu_wall) for g in b.geoms]
    p = params(n_it=n_it)
    v0 = np.random.default_rng(seed).uniform(-vmax, vmax, (n, 3)).astype(np.float32)
    return b.x, b.r, geoms, p, dict(resort_every=resort_every, v=v0, **kw)


def gpu_bed(x, r, geoms, p, extra, theta=THETA):
    q = dict(p)
    q.update(kn_scale=theta[0], mu_t=theta[1], mu_r=theta[2])
    extra = dict(extra)
    v0 = extra.pop("v", None)
    return make_gpu(x, r, q, geoms, v=v0, **extra)


def gpu_objective(x, r, geoms, p, extra, theta, steps, W):
    bed = gpu_bed(x, r, geoms, p, extra, theta)
    F = bed.record(steps, 4)
    bed.close()
    return float((F * W).sum())


def weights(steps, ng=6, seed=3):
    return np.random.default_rng(seed).normal(size=(steps, ng, 3))


def oracle_gradient(x, r, geoms, p, steps, W, v0):
    op = OracleParams(**p)
    st = ts.TorchStepper(op, np.asarray(r, np.float64), np.arange(len(r), dtype=np.int32), oracle_geoms(geoms))
    th = [torch.tensor(float(np.float32(v)), dtype=torch.float64, requires_grad=True) for v in THETA]
    xx = torch.as_tensor(x, dtype=torch.float64)
    v = torch.as_tensor(np.asarray(v0, np.float64))
    w = torch.zeros_like(xx)
    warm = {}
    pp = [torch.tensor(g.c, dtype=torch.float64) for g in oracle_geoms(geoms)]
    J = torch.zeros((), dtype=torch.float64)
    for t in range(steps):
        xx, v, w, warm, F, pp = st.step(xx, v, w, th, warm, pp)
        J = J + (torch.as_tensor(W[t]) * F).sum()
    J.backward()
    return float(J.detach()), np.array([float(t.grad) for t in th])


@pytest.mark.parametrize("mu_wall,lanes", [(0.0, 0), (0.3, 2)])
def test_adjoint_matches_fp64_oracle_gradient(mu_wall, lanes):
    steps = 10
    x, r, geoms, p, extra = small_cell(mu_wall=mu_wall, lanes=lanes)
    W = weights(steps)
    bed = gpu_bed(x, r, geoms, p, extra)
    F = bed.record(steps, 4)          # segments of 4, 4, 2 steps
    g = bed.adjoint(W)
    J = float((F * W).sum())
    Jo, go = oracle_gradient(x, r, geoms, p, steps, W, extra["v"])
    assert abs(J - Jo) <= 1e-4 * np.abs(F * W).sum()
    scale = np.abs(go).max()
    assert np.all(np.abs(go) > 1e-3 * scale), go   # every parameter matters in this case
    assert np.all(np.abs(g - go) <= 2e-4 * scale), (g, go)


def test_adjoint_matches_central_differences():
    steps = 12
    x, r, geoms, p, extra = small_cell(n=200, n_it=40)
    W = weights(steps)
    bed = gpu_bed(x, r, geoms, p, extra)
    bed.record(steps, 5)
    g = bed.adjoint(W)
    fd = np.zeros(3)
    for k in range(3):
        h = 1e-3 * THETA[k]
        tp, tm = list(THETA), list(THETA)
        tp[k] += h
        tm[k] -= h
        fd[k] = (gpu_objective(x, r, geoms, p, extra, tp, steps, W) -
                 gpu_objective(x, r, geoms, p, extra, tm, steps, W)) / (2 * h)
    assert np.all(np.abs(fd) > 1e-3 * np.abs(fd).max()), fd
    assert np.all(np.abs(g - fd) <= 5e-3 * np.abs(fd).max()), (g, fd)


def test_checkpoint_interval_does_not_change_the_gradient():
    steps = 9
    x, r, geoms, p, extra = small_cell()
    W = weights(steps)
    grads, forces = [], []
    for every in (1, 4, 9, 50):
        bed = gpu_bed(x, r, geoms, p, extra)
        forces.append(bed.record(steps, every))
        grads.append(bed.adjoint(W))
        grads.append(bed.adjoint(W))   # repeatable on the same recording
        bed.close()
    for F in forces[1:]:
        assert np.array_equal(F, forces[0])
    for g in grads[1:]:
        assert np.array_equal(g, grads[0])


def test_record_forces_equal_stepping_and_state_is_restored():
    steps = 7
    x, r, geoms, p, extra = small_cell()
    a = gpu_bed(x, r, geoms, p, extra)
    b = gpu_bed(x, r, geoms, p, extra)
    F = a.record(steps, 3)
    for t in range(steps):
        b.step(1)
        for gi in range(6):
            assert np.array_equal(b.read_forces(gi)[0], F[t, gi])
    a.adjoint(weights(steps))
    # the adjoint leaves the bed after the window: it continues like b
    for gi in range(6):
        assert np.array_equal(a.read_forces(gi)[0], b.read_forces(gi)[0])
    a.step(5)
    b.step(5)
    for u, v in zip(a.read_state(), b.read_state()):
        assert np.array_equal(u, v)


def test_autograd_function_and_deviatoric_stress():
    from paper_2501_05300_gb300.adjoint import CellGeometry, deviatoric_stress, geom_forces
    steps = 8
    x, r, geoms, p, extra = small_cell()
    bed = gpu_bed(x, r, geoms, p, extra)
    cell = CellGeometry.from_bed(bed)
    theta = torch.tensor(THETA, dtype=torch.float64, requires_grad=True)
    F = geom_forces(bed, theta, steps, ckpt_every=3)
    J = deviatoric_stress(F, cell).mean()
    J.backward()
    # the same functional through the C call with explicit weights
    Fw = F.detach().clone().requires_grad_(True)
    deviatoric_stress(Fw, cell).mean().backward()
    g = bed.adjoint(Fw.grad.numpy())
    assert np.array_equal(theta.grad.numpy(), g)
    assert np.isfinite(float(J.detach()))
    assert np.all(np.isfinite(g)) and np.abs(g).max() > 0


def test_adjoint_errors():
    from paper_2501_05300_gb300.dem import DEM_ERR_ARG, DEM_ERR_STATE, DemError
    x, r, geoms, p, extra = small_cell()
    bed = gpu_bed(x, r, geoms, p, extra)
    with pytest.raises(DemError) as e:
        bed.adjoint(weights(3))
    assert e.value.status == DEM_ERR_STATE
    bed.record(3, 2)
    bed.step(1)
    with pytest.raises(DemError) as e:
        bed.adjoint(weights(3))
    assert e.value.status == DEM_ERR_STATE
    spinning = beds.GeomSpec(beds.BOX, (0.0, 0.0, -1.0), he=(0.1, 0.1, 0.1), w=(0.0, 0.0, 1.0))
    other = gpu_bed(x, r, list(geoms) + [spinning], p, extra)
    with pytest.raises(DemError) as e:
        other.record(2, 1)
    assert e.value.status == DEM_ERR_ARG


def test_checkpoint_restore_repeats_steps_bitwise():
    x, r, geoms, p, extra = small_cell()
    bed = gpu_bed(x, r, geoms, p, extra)
    bed.step(4)
    h = bed.save_checkpoint()
    bed.step(6)
    s1 = bed.read_state()
    f1 = bed.read_forces(1)[0]
    bed.restore_checkpoint(h)
    bed.step(6)
    for u, v in zip(bed.read_state(), s1):
        assert np.array_equal(u, v)
    assert np.array_equal(bed.read_forces(1)[0], f1)
    # a restore keeps settings changed since the save
    bed.restore_checkpoint(h)
    bed.set_material(mu_t=0.25)
    bed.step(6)
    assert not np.array_equal(bed.read_state()[1], s1[1])
    bed.free_checkpoint(h)


def primitive_case(n_it=30, seed=19):
    x, r, geoms = primitive_cloud()
    p = params(n_it=n_it)
    v0 = np.random.default_rng(seed).uniform(-0.05, 0.05, (len(r), 3)).astype(np.float32)
    return x, r, geoms, p, dict(resort_every=3, v=v0)


def primitive_weights(steps, ng, seed=4):
    W = np.zeros((steps, ng, 3))
    W[:, 5:7] = np.random.default_rng(seed).normal(size=(steps, 2, 3))   # the box and the cylinder
    return W


def test_adjoint_with_boxes_and_cylinders_matches_fp64_oracle():
    """Forces on a translating oblique box and a tilted cylinder pressed into a
    cloud (contacts on faces, edges, corners, caps, sides and rims): the
    normal moves with the sphere off the faces, and the gradient must follow."""
    steps = 8
    x, r, geoms, p, extra = primitive_case()
    W = primitive_weights(steps, len(geoms))
    bed = gpu_bed(x, r, geoms, p, extra)
    F = bed.record(steps, 3)
    g = bed.adjoint(W)
    J = float((F * W).sum())
    Jo, go = oracle_gradient(x, r, geoms, p, steps, W, extra["v"])
    assert abs(J - Jo) <= 1e-4 * np.abs(F * W).sum()
    scale = np.abs(go).max()
    assert scale > 0
    assert np.all(np.abs(g - go) <= 2e-4 * scale), (g, go)


def test_adjoint_with_boxes_and_cylinders_matches_central_differences():
    steps = 8
    x, r, geoms, p, extra = primitive_case(n_it=40)
    W = primitive_weights(steps, len(geoms))
    bed = gpu_bed(x, r, geoms, p, extra)
    bed.record(steps, 4)
    g = bed.adjoint(W)
    fd = np.zeros(3)
    for k in range(3):
        h = 1e-3 * THETA[k]
        tp, tm = list(THETA), list(THETA)
        tp[k] += h
        tm[k] -= h
        fd[k] = (gpu_objective(x, r, geoms, p, extra, tp, steps, W) -
                 gpu_objective(x, r, geoms, p, extra, tm, steps, W)) / (2 * h)
    assert np.abs(fd).max() > 0
    assert np.all(np.abs(g - fd) <= 5e-3 * np.abs(fd).max()), (g, fd)
