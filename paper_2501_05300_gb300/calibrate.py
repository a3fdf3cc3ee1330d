"""Calibration of the contact parameters against bulk targets with the
adjoint's gradients (Gauss-Newton).

theta = (k_n scale, mu_t, mu_r) (Sec. 2.2, Eqs. 6-7).  Each residual is a
functional of a window of steps of one bed; its gradient in theta comes from
the library's hand-written adjoint (adjoint.geom_forces), taken along the
contact topology of every step of the window.

The target used here is the triaxial friction angle of the paper's beds
(Sec. 3.2, Table 1): at confining stress sigma_3 a sample fails when
sigma_1 = K sigma_3, K = (1 + sin phi) / (1 - sin phi) (Mohr-Coulomb, no
cohesion, as for the paper's dry sand).  One cell per confining stress is
consolidated, then sheared with the candidate theta to the axial strain of
its peak; the residual is the mean over a window there of
(sigma_1 - K sigma_3) / sigma_3, the side walls held and the platen still
shearing during the window.
Because every evaluation re-shears the cell with the candidate theta, the
sample's fabric belongs to that theta, and the Gauss-Newton iteration stops
where the re-sheared peak meets the target.  The gradient is the derivative
at fixed history (the window only): it steers the step, and convergence is
judged on the residuals themselves.
"""
from __future__ import annotations

import numpy as np
import torch

from . import beds, triaxial
from .adjoint import CellGeometry, geom_forces, principal_stresses


def gauss_newton_step(r, J, damping=0.0):
    """The step d minimising |r + J d|^2 + damping |diag(J^T J)^(1/2) d|^2
    (Levenberg-Marquardt scaling): (J^T J + damping diag(J^T J)) d = -J^T r."""
    r = np.asarray(r, np.float64).reshape(-1)
    J = np.asarray(J, np.float64).reshape(r.size, -1)
    A = J.T @ J
    A = A + damping * np.diag(np.diag(A))
    return -np.linalg.solve(A, J.T @ r)


class FailureWindow:
    """Residual of one triaxial cell at confining stress sigma3.

    bed: a Bed holding the cell (its first six primitives are the walls),
    consolidated to sigma3 and saved in `consolidated` (a checkpoint).  For a
    candidate theta the cell is restored, given theta, sheared with servoed
    side walls to `strain` (triaxial.shear), and then `steps` steps are
    recorded with the side walls held and the platen still moving; the
    residual is the window mean of (sigma_1 - K sigma_3) / sigma3."""

    def __init__(self, bed, consolidated, sigma3, K, strain, steps, rate=0.5, ckpt_every=20, reshear=True):
        self.bed, self.start, self.sigma3, self.K = bed, consolidated, float(sigma3), float(K)
        self.strain, self.steps, self.rate, self.every = float(strain), int(steps), float(rate), int(ckpt_every)
        self.reshear = reshear
        self.last = {}

    def _window_start(self, theta):
        b = self.bed
        b.restore_checkpoint(self.start)
        b.set_material(kn_scale=float(theta[0]), mu_t=float(theta[1]), mu_r=float(theta[2]))
        if self.reshear and self.strain > 0:
            triaxial.shear(b, self.sigma3, self.rate, self.strain)

    def evaluate(self, theta, grad=True):
        """(residual, d residual / d theta (3,) or None)."""
        self._window_start(theta)
        cell = CellGeometry.from_bed(self.bed)
        th = torch.tensor([float(t) for t in theta], dtype=torch.float64, requires_grad=grad)
        F = geom_forces(self.bed, th, self.steps, self.every)
        s1, s3 = principal_stresses(F, cell)
        J = ((s1 - self.K * s3) / self.sigma3).mean()
        g = None
        if grad:
            J.backward()
            g = th.grad.numpy().copy()
        self.last = dict(sigma1=float(s1.detach().mean()), sigma3=float(s3.detach().mean()))
        return float(J.detach()), g


class MatchWindow:
    """Residual of a cell against a target mean deviatoric stress [Pa] (the
    refined cell against the fine cell's response, the same protocol): the
    window mean of sigma_1 - sigma_3 over `steps` steps from the saved state
    `start`, minus the target, over the target."""

    def __init__(self, bed, start, target, steps, ckpt_every=20):
        self.bed, self.start, self.target = bed, start, float(target)
        self.steps, self.every = int(steps), int(ckpt_every)
        self.last = {}

    def evaluate(self, theta, grad=True):
        b = self.bed
        b.restore_checkpoint(self.start)
        cell = CellGeometry.from_bed(b)
        th = torch.tensor([float(t) for t in theta], dtype=torch.float64, requires_grad=grad)
        F = geom_forces(b, th, self.steps, self.every)
        s1, s3 = principal_stresses(F, cell)
        J = ((s1 - s3).mean() - self.target) / abs(self.target)
        g = None
        if grad:
            J.backward()
            g = th.grad.numpy().copy()
        self.last = dict(sigma1=float(s1.detach().mean()), sigma3=float(s3.detach().mean()))
        return float(J.detach()), g


def calibrate(windows, theta0, free=(1, 2), max_iter=8, tol=5e-3, damping=1e-3,
              bounds=((0.25, 4.0), (0.02, 2.0), (0.0, 1.0))):
    """Gauss-Newton on the free components of theta until every |residual| <=
    tol (or max_iter).  Returns (theta, history); history[k] holds theta, the
    residuals, their Jacobian on the free components and each window's mean
    stresses."""
    theta = np.array(theta0, np.float64)
    free = list(free)
    hist = []
    for _ in range(max_iter):
        r, J, st = [], [], []
        for w in windows:
            v, g = w.evaluate(theta)
            r.append(v)
            J.append(g[free])
            st.append(dict(w.last))
        r, J = np.array(r), np.array(J)
        hist.append(dict(theta=theta.tolist(), residuals=r.tolist(), jacobian=J.tolist(), stresses=st))
        if np.abs(r).max() <= tol:
            break
        d = gauss_newton_step(r, J, damping)
        for k, i in enumerate(free):
            theta[i] = float(np.clip(theta[i] + d[k], bounds[i][0], bounds[i][1]))
    return theta, hist


def friction_angle(windows):
    """Friction angle [deg] and cohesion [Pa] of the windows' last evaluated
    mean states, by the Mohr-Coulomb fit (triaxial.mohr_coulomb_fit)."""
    s3 = [w.last["sigma3"] for w in windows]
    s1 = [w.last["sigma1"] for w in windows]
    return triaxial.mohr_coulomb_fit(s3, s1)


def consolidated_cell(dem, n, sigma3, seed=2505, lanes=0, material=None, **cell_kw):
    """A triaxial cell of n spheres (beds.triaxial_cell) consolidated to sigma3
    with the generation friction of Sec. 3.1 (mu_t 0.1, mu_r 0.01), no gravity,
    dt 5e-5 s and 60 sweeps; then switched to the test settings (dt 1e-5 s,
    N_it from Eq. 8 with n_d = h / d) and saved.  Returns (bed, checkpoint)."""
    from . import rules
    spec = beds.triaxial_cell(n, seed=seed, **cell_kw)
    m = material or spec.material
    bed = dem.Bed(spec.x, spec.r, geoms=spec.geoms, rho=m.rho, mu_t=0.1, mu_r=0.01, n_it=60, dt=5e-5,
                  gravity=(0.0, 0.0, 0.0), lanes=lanes)
    triaxial.consolidate(bed, sigma3)
    _, L = triaxial.wall_stress(bed)
    d = 2.0 * float(np.mean(spec.r))
    nit = rules.n_iterations(rules.network_length_uniform(float(L[2]), d), 0.02)
    bed.set_params(dt=1e-5, n_it=nit, mu_t=m.mu_t, mu_r=m.mu_r, gravity=(0.0, 0.0, 0.0), lanes=lanes)
    bed.step(20)
    return bed, bed.save_checkpoint()
