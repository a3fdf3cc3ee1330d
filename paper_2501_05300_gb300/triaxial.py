"""Box triaxial test (Sec. 3.2) on a bed of this library, and the Mohr-Coulomb
failure line fitted to its peak states.

The cell is the bed's first six primitives, frictionless planar walls
(beds.cell_walls): floor, platen and four side walls.  Consolidation: every
wall moves along its inward normal at a speed proportional to the gap between
its normal stress and the confining stress sigma_3 until all six hold it.
Shearing: the platen moves down at a constant axial strain rate while the
side walls keep servoing to sigma_3 (a drained test with constant minor
stress).  The servo acts between steps, outside the solve.

The bulk friction angle phi and cohesion c follow from the peak states
(sigma_3, sigma_1) at several confining stresses: the Mohr circles with those
principal stresses touch the failure line tau = c + sigma tan(phi) exactly when
sigma_1 = K sigma_3 + 2 c sqrt(K), K = (1 + sin phi) / (1 - sin phi), so a
least-squares line through the peak states gives K and c (Sec. 3.2 fits the
circles of minor stress sigma_3 and peak deviatoric stress sigma_1 - sigma_3).
"""
from __future__ import annotations

import math

import numpy as np

from . import beds

SIDE_WALLS = (beds.WALL_XLO, beds.WALL_XHI, beds.WALL_YLO, beds.WALL_YHI)


def K_of_phi(phi_deg: float) -> float:
    """Passive ratio sigma_1 / sigma_3 at failure for friction angle phi."""
    s = math.sin(math.radians(phi_deg))
    return (1.0 + s) / (1.0 - s)


def phi_of_K(K: float) -> float:
    """Friction angle [deg] of a failure ratio K = sigma_1 / sigma_3 (no cohesion)."""
    return math.degrees(math.asin((K - 1.0) / (K + 1.0)))


def mohr_coulomb_fit(sigma3, sigma1):
    """Friction angle [deg] and cohesion [Pa] of the failure line through peak
    states (sigma_3, sigma_1): least squares of sigma_1 = K sigma_3 + b, then
    sin phi = (K - 1) / (K + 1) and c = b / (2 sqrt K).  With one state the
    line goes through the origin (c = 0)."""
    s3 = np.asarray(sigma3, np.float64).reshape(-1)
    s1 = np.asarray(sigma1, np.float64).reshape(-1)
    if s3.size != s1.size or s3.size == 0:
        raise ValueError("need as many sigma_1 as sigma_3 values, at least one")
    if s3.size == 1:
        K, b = float(s1[0] / s3[0]), 0.0
    else:
        A = np.stack([s3, np.ones_like(s3)], 1)
        (K, b), *_ = np.linalg.lstsq(A, s1, rcond=None)
        K, b = float(K), float(b)
    if not K > 1.0:
        raise ValueError(f"failure ratio K = {K} <= 1: not a frictional failure line")
    return phi_of_K(K), b / (2.0 * math.sqrt(K))


def wall_stress(bed, walls=range(6)):
    """Normal stress on each wall [Pa] (compression positive) in the last
    step, and the cell's edge lengths (x, y, z)."""
    c = [np.array(bed.read_geom(g).c[:]) for g in range(6)]
    lo = np.array([c[beds.WALL_XLO][0], c[beds.WALL_YLO][1], c[beds.FLOOR][2]])
    hi = np.array([c[beds.WALL_XHI][0], c[beds.WALL_YHI][1], c[beds.PLATEN][2]])
    L = hi - lo
    area = {beds.FLOOR: L[0] * L[1], beds.PLATEN: L[0] * L[1], beds.WALL_XLO: L[1] * L[2],
            beds.WALL_XHI: L[1] * L[2], beds.WALL_YLO: L[0] * L[2], beds.WALL_YHI: L[0] * L[2]}
    out = {}
    for g in walls:
        nrm = np.array(bed.geoms[g].R)[[2, 5, 8]]     # inward normal
        f = bed.read_forces(g)[0]
        out[g] = float(-(f @ nrm) / area[g])
    return out, L


def servo(bed, walls, target, vmax):
    """Move each wall along its inward normal at vmax (target - sigma) / target,
    clipped to +-vmax; returns the stresses it acted on."""
    sig, L = wall_stress(bed, walls)
    for g in walls:
        nrm = np.array(bed.geoms[g].R)[[2, 5, 8]]
        u = vmax * float(np.clip((target - sig[g]) / target, -1.0, 1.0))
        bed.apply_plate_velocity(g, tuple(u * nrm))
    return sig, L


def hold(bed, walls=range(6)):
    for g in walls:
        bed.apply_plate_velocity(g, (0.0, 0.0, 0.0))


def consolidate(bed, sigma3, vmax=0.05, tol=0.03, chunk=10, max_steps=8000, settled_chunks=10):
    """Isotropic consolidation: all six walls servo to sigma3 until every wall
    is within tol of it for `settled_chunks` chunks in a row (or max_steps).
    The walls are held when it returns.  Returns the steps taken."""
    steps, ok = 0, 0
    while steps < max_steps:
        sig, _ = servo(bed, range(6), sigma3, vmax)
        bed.step(chunk)
        steps += chunk
        ok = ok + 1 if all(abs(v - sigma3) < tol * sigma3 for v in sig.values()) else 0
        if ok >= settled_chunks:
            break
    hold(bed)
    return steps


def shear(bed, sigma3, rate, strain, chunk=20, vmax=0.05):
    """Drained shearing: the platen moves down at `rate` (axial strain per
    second, of the current height) while the side walls servo to sigma3,
    until the axial strain reaches `strain`.  Returns the samples
    (axial strain, sigma_1, sigma_3) taken every chunk.  When it returns the
    side walls are held and the platen keeps moving, so the steps that follow
    go on shearing the sample (a window to differentiate, in which no wall is
    servoed)."""
    sig, L = wall_stress(bed)
    h0 = float(L[2])
    out = []
    while True:
        sig, L = servo(bed, SIDE_WALLS, sigma3, vmax)
        e = 1.0 - float(L[2]) / h0
        s3 = float(np.mean([sig[g] for g in SIDE_WALLS]))
        s1 = wall_stress(bed, (beds.PLATEN,))[0][beds.PLATEN]
        out.append((e, s1, s3))
        bed.apply_plate_velocity(beds.PLATEN, (0.0, 0.0, -rate * float(L[2])))
        if e >= strain:
            break
        bed.step(chunk)
    hold(bed, SIDE_WALLS)
    return np.array(out)


def peak_state(samples):
    """(sigma_3, sigma_1) at the largest deviatoric stress of a shear record."""
    s = np.asarray(samples)
    k = int(np.argmax(s[:, 1] - s[:, 2]))
    return float(s[k, 2]), float(s[k, 1])
