"""Gradients of geometry forces with respect to the contact parameters.

`geom_forces(bed, theta, nsteps)` advances the bed nsteps steps with
theta = (k_n scale, mu_t, mu_r) and returns the force on every primitive in
every step as a tensor that autograd differentiates with respect to theta:
the backward pass is the library's hand-written adjoint of the step
(dem_step_adjoint), along the contact set of every step, with the window
recomputed from checkpoints taken every `ckpt_every` steps (0: the interval
that minimises memory, chosen by the library).

`deviatoric_stress` turns the wall forces of a box triaxial cell (Sec. 3.2)
into sigma_1 - sigma_3 per step, so that, for instance,

    F = geom_forces(bed, theta, 400)
    J = deviatoric_stress(F, cell).mean()
    J.backward()          # theta.grad = dJ / d(k_n scale, mu_t, mu_r)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import beds as _beds


class GeomForces(torch.autograd.Function):
    """theta (3,) -> forces (nsteps, n_geom, 3), float64, on the CPU."""

    @staticmethod
    def forward(ctx, theta, bed, nsteps, ckpt_every):
        kn_scale, mu_t, mu_r = (float(t) for t in theta.detach().cpu().reshape(3))
        bed.set_material(kn_scale=kn_scale, mu_t=mu_t, mu_r=mu_r)
        F = bed.record(nsteps, ckpt_every)
        ctx.bed = bed
        ctx.theta_dtype = theta.dtype
        ctx.theta_device = theta.device
        return torch.from_numpy(F)

    @staticmethod
    def backward(ctx, grad_F):
        g = ctx.bed.adjoint(grad_F.detach().to(torch.float64).cpu().contiguous().numpy())
        return torch.as_tensor(g, dtype=ctx.theta_dtype, device=ctx.theta_device), None, None, None


def geom_forces(bed, theta, nsteps, ckpt_every=0):
    """Forces on the bed's primitives over nsteps steps, differentiable in theta.
    The bed is left after the window; each call continues from where it is."""
    return GeomForces.apply(theta, bed, int(nsteps), int(ckpt_every))


@dataclass
class CellGeometry:
    """Wall positions of a box triaxial cell at the start of a window and the
    platen's speed (the walls indexed as in beds.cell_walls)."""
    lo: np.ndarray      # (x, y, z) of the low walls (x, y side walls; floor)
    hi: np.ndarray      # (x, y, z) of the high walls (platen z)
    v: np.ndarray       # (6, 3) wall velocities
    dt: float

    @classmethod
    def from_bed(cls, bed):
        c = [np.array(bed.read_geom(g).c[:]) for g in range(6)]
        v = np.array([bed.read_geom(g).v[:] for g in range(6)])
        lo = np.array([c[_beds.WALL_XLO][0], c[_beds.WALL_YLO][1], c[_beds.FLOOR][2]])
        hi = np.array([c[_beds.WALL_XHI][0], c[_beds.WALL_YHI][1], c[_beds.PLATEN][2]])
        return cls(lo, hi, v, bed.dt)


def principal_stresses(F, cell: CellGeometry):
    """(sigma_1, sigma_3) in every step [Pa]: sigma_1 the platen's normal force
    over its area, sigma_3 the mean normal stress on the four side walls, with
    the walls where they stand in that step (they move kinematically)."""
    steps = F.shape[0]
    t = torch.arange(steps, dtype=F.dtype)[:, None]
    lo = torch.as_tensor(cell.lo, dtype=F.dtype) + t * cell.dt * torch.as_tensor(
        [cell.v[_beds.WALL_XLO][0], cell.v[_beds.WALL_YLO][1], cell.v[_beds.FLOOR][2]], dtype=F.dtype)
    hi = torch.as_tensor(cell.hi, dtype=F.dtype) + t * cell.dt * torch.as_tensor(
        [cell.v[_beds.WALL_XHI][0], cell.v[_beds.WALL_YHI][1], cell.v[_beds.PLATEN][2]], dtype=F.dtype)
    L = hi - lo
    a_z = L[:, 0] * L[:, 1]
    a_x = L[:, 1] * L[:, 2]
    a_y = L[:, 0] * L[:, 2]
    s1 = F[:, _beds.PLATEN, 2] / a_z
    s3 = 0.25 * ((F[:, _beds.WALL_XHI, 0] - F[:, _beds.WALL_XLO, 0]) / a_x +
                 (F[:, _beds.WALL_YHI, 1] - F[:, _beds.WALL_YLO, 1]) / a_y)
    return s1, s3


def deviatoric_stress(F, cell: CellGeometry):
    """sigma_1 - sigma_3 in every step [Pa] (see principal_stresses)."""
    s1, s3 = principal_stresses(F, cell)
    return s1 - s3
