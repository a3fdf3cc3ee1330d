"""Seeded synthetic inputs: particle beds and the rigid geometry around them.

Only input construction lives here (positions, radii, walls, plates); none of
the contact law, solver or integrator.  Beds follow the paper's recipe
(Sec. 3.1): layers of particles whose diameter is uniform in [0.9, 1.1] of the
layer's nominal size, coarser layers below finer ones (Sec. 2.1).  Instead of
emitting and relaxing particles, each layer starts as a jittered face-centred
cubic lattice with a small gap between neighbours, which settling under
gravity compacts to a dense packing.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

PLANE, BOX, CYLINDER = 0, 1, 2
IDENT = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)

# dry-sand material of the paper (Sec. 3.1); density and friction as overridden
# by the workloads below where they state their own values
RHO_PAPER, E_PAPER, NU_PAPER, MU_T_PAPER, MU_R_PAPER = 2200.0, 1e9, 0.15, 0.3, 0.02


@dataclass
class GeomSpec:
    """A rigid, kinematic primitive.  R is row-major; column k is local axis k.
    plane: c a point on it, normal = local z (solid below);
    box: c centre, he half extents; cylinder: c centre, axis local z,
    he[0] radius, he[2] half height."""
    type: int
    c: tuple
    R: tuple = IDENT
    he: tuple = (0.0, 0.0, 0.0)
    v: tuple = (0.0, 0.0, 0.0)
    w: tuple = (0.0, 0.0, 0.0)
    E: float = E_PAPER
    nu: float = NU_PAPER
    mu_t: float = 0.5
    mu_r: float = 0.02


@dataclass
class Material:
    rho: float = 2600.0
    E: float = E_PAPER
    nu: float = NU_PAPER
    mu_t: float = 0.5
    mu_r: float = 0.02


@dataclass
class Bed:
    """Particles (x float64 [N,3], r float32 [N], ids 0..N-1) plus geometry."""
    x: np.ndarray
    r: np.ndarray
    geoms: list = field(default_factory=list)
    material: Material = field(default_factory=Material)
    name: str = ""
    plate: int = -1                  # index of the driven plate primitive, -1 none
    plate_parts: tuple = ()          # primitives moved together with the plate
    box: tuple = (0.0, 0.0, 0.0)     # container extents

    @property
    def n(self) -> int:
        return int(self.r.shape[0])

    def v(self):
        return np.zeros((self.n, 3), np.float32)


def plane(point, normal, mu_t=0.0, mu_r=0.0):
    """Plane through `point` whose outward normal is `normal` (solid behind it)."""
    nz = np.asarray(normal, float)
    nz = nz / np.linalg.norm(nz)
    a = np.array([1.0, 0, 0]) if abs(nz[0]) < 0.9 else np.array([0, 1.0, 0])
    nx = a - (a @ nz) * nz
    nx /= np.linalg.norm(nx)
    ny = np.cross(nz, nx)
    Rm = np.stack([nx, ny, nz], axis=1)
    return GeomSpec(PLANE, tuple(map(float, point)), tuple(Rm.reshape(-1)), mu_t=mu_t, mu_r=mu_r)


def open_box_walls(lx, ly, mu_wall=0.0):
    """Floor z=0 and four side walls of [0,lx]x[0,ly]; frictionless walls as in
    the paper's containers (Sec. 3.1 and 3.3)."""
    return [plane((0, 0, 0), (0, 0, 1), mu_wall, mu_wall),
            plane((0, 0, 0), (1, 0, 0), mu_wall, mu_wall),
            plane((lx, 0, 0), (-1, 0, 0), mu_wall, mu_wall),
            plane((0, 0, 0), (0, 1, 0), mu_wall, mu_wall),
            plane((0, ly, 0), (0, -1, 0), mu_wall, mu_wall)]


def _uniform_radii(rng, r_nom, n, spread):
    return (r_nom * rng.uniform(1.0 - spread, 1.0 + spread, n)).astype(np.float32)


def lattice_layer(rng, lx, ly, z0, n_target, r_nom, spread=0.1, gap=0.03, margin=None):
    """n_target spheres of radius r_nom*U[1-spread,1+spread] on a jittered
    face-centred cubic lattice (triangular layers stacked ABC) inside
    [0,lx]x[0,ly], layers stacked upwards from z0.  The nearest-neighbour
    distance leaves a gap so that no two spheres overlap.  Returns (x, r, z_top)."""
    rmax = r_nom * (1 + spread)
    a = 2 * rmax * (1 + gap)                 # nearest-neighbour distance
    jit = 0.45 * (a - 2 * rmax)
    margin = rmax * 1.001 + jit if margin is None else margin
    dy, dz = a * math.sqrt(3.0) / 2.0, a * math.sqrt(2.0 / 3.0)
    pts, k = [], 0
    count = 0
    while count < n_target:
        sx, sy = (k % 3) * a / 2.0, (k % 3) * a * math.sqrt(3.0) / 6.0
        ys = np.arange(margin + sy, ly - margin + 1e-12, dy)
        rows = []
        for j, y in enumerate(ys):
            xs = np.arange(margin + sx + (a / 2.0 if j % 2 else 0.0), lx - margin + 1e-12, a)
            rows.append(np.stack([xs, np.full_like(xs, y), np.full_like(xs, z0 + margin + k * dz)], 1))
        layer = np.concatenate(rows) if rows else np.zeros((0, 3))
        pts.append(layer)
        count += len(layer)
        k += 1
        if k > 100000:
            raise ValueError("footprint too small for one sphere")
    x = np.concatenate(pts)[:n_target]
    x = x + rng.uniform(-jit, jit, x.shape)
    r = _uniform_radii(rng, r_nom, len(x), spread)
    return x.astype(np.float64), r, z0 + margin + (k - 1) * dz + rmax * 1.001 + jit


def layered_bed(lx, ly, layers_bottom_up, spread=0.1, phi=0.636, seed=0, gap=0.03):
    """Layers (r_nominal, settled_thickness) from the bottom up.  Each layer
    holds round(lx ly thickness phi / <V>) spheres, <V> the mean sphere volume
    of its radius distribution; the lattice is a little looser than phi and
    settles."""
    rng = np.random.default_rng(seed)
    xs, rs, z = [], [], 0.0
    for r_nom, thick in layers_bottom_up:
        # <r^3> of r_nom*U[1-s,1+s] is r_nom^3 ((1+s)^4-(1-s)^4)/(8s)
        m3 = r_nom ** 3 * (((1 + spread) ** 4 - (1 - spread) ** 4) / (8 * spread) if spread > 0 else 1.0)
        vmean = 4.0 / 3.0 * math.pi * m3
        n_target = int(round(lx * ly * thick * phi / vmean))
        if n_target == 0:
            continue
        x, r, z = lattice_layer(rng, lx, ly, z, n_target, r_nom, spread, gap)
        xs.append(x)
        rs.append(r)
    return np.concatenate(xs), np.concatenate(rs)


# --------------------------------------------------------------------------- #
# the workloads                                                               #
# --------------------------------------------------------------------------- #
def settling_box(n=2000, seed=2502):
    """2,000 spheres, r ~ U[5,6] mm, in a 0.1 x 0.1 x 0.3 m box on a jittered
    lattice (spacing 12.5 mm); settles under gravity (rho 2600, mu 0.5)."""
    rng = np.random.default_rng(seed)
    s, lx = 12.5e-3, 0.1
    per_side = int(math.floor((lx - 12e-3) / s)) + 1
    per = per_side * per_side
    idx = np.arange(n)
    ix, iy, iz = idx % per_side, (idx // per_side) % per_side, idx // per
    x = np.stack([6.22e-3 + ix * s, 6.22e-3 + iy * s, 6.22e-3 + iz * s], axis=1).astype(np.float64)
    x += rng.uniform(-0.2e-3, 0.2e-3, x.shape)
    r = rng.uniform(5e-3, 6e-3, n).astype(np.float32)
    mat = Material(rho=2600.0, mu_t=0.5, mu_r=0.02)
    return Bed(x, r, open_box_walls(lx, lx), mat, name=f"settling box, {n} spheres r~U[5,6] mm",
               box=(lx, lx, 0.3))


def refined_layers(top_r=2.5e-3, top_thickness=0.02, growth=2.0, n_coarser=3, depth=0.25):
    """Layer list (bottom up) of a refined bed: top layer r = top_r, thickness
    top_thickness = eta d_0; each layer below doubles r and its thickness
    (d_n = r d_{n-1}, thickness eta d_n, Sec. 2.1); the coarsest fills the rest."""
    eta = top_thickness / (2 * top_r)
    tops = []
    r, z = top_r, 0.0
    for i in range(n_coarser + 1):
        t = eta * 2 * r
        if i == n_coarser:
            t = depth - z
        tops.append((r, t))
        z += t
        r *= growth
    return list(reversed(tops))


def graded_layers(top_r, top_thickness, growth, cap_ratio=8.0, depth=0.25):
    """Layers (bottom up) of a bed refined from the top: the top layer has
    radius top_r and thickness eta d_0 = top_thickness; below it every layer's
    radius grows by `growth` (d_n = r d_{n-1}) and its thickness is eta d_n
    (Sec. 2.1), the radius capped at cap_ratio * top_r; the capped size fills
    the rest of the depth."""
    eta = top_thickness / (2 * top_r)
    cap = cap_ratio * top_r
    out, r, z = [], top_r, 0.0
    while True:
        t = eta * 2 * r
        if r >= cap * (1 - 1e-9) or z + t >= depth - 1e-12:
            out.append((r, depth - z))
            break
        out.append((r, t))
        z += t
        r = min(r * growth, cap)
    return list(reversed(out))


def natural_density(layers, spread=0.1, phi=0.636):
    """Particles per square metre of footprint of a layer list."""
    tot = 0.0
    for r, t in layers:
        m3 = r ** 3 * ((1 + spread) ** 4 - (1 - spread) ** 4) / (8 * spread)
        tot += t * phi / (4.0 / 3.0 * math.pi * m3)
    return tot


BATCH_DEPTHS = (0.01, 0.02, 0.03, 0.04, 0.06, 0.08)
BATCH_GROWTHS = (1.25, 1.5, 1.75, 2.0, 2.5, 3.0)


def batch_specs(n_min=20_000, n_max=500_000, depth=0.25, r0=2.5e-3):
    """The 6 x 6 grid of refinement depth x radius growth: for each bed its
    layers, the footprint side that gives its particle count, and N_it from
    Eqs. 8 and 10.  Counts are log-spaced from n_min to n_max in the order of
    the beds' natural densities."""
    combos = [(dd, g, graded_layers(r0, dd, g, depth=depth)) for dd in BATCH_DEPTHS for g in BATCH_GROWTHS]
    dens = [natural_density(l) for _, _, l in combos]
    order = sorted(range(len(combos)), key=lambda k: dens[k])
    counts = np.geomspace(n_min, n_max, len(combos))
    out = [None] * len(combos)
    for rank, k in enumerate(order):
        dd, g, layers = combos[k]
        side = math.sqrt(counts[rank] / dens[k])
        eta = dd / (2 * r0)
        d_min, d_max = 2 * r0, 2 * max(r for r, _ in layers)
        zmax = sum(t for r, t in layers if r < max(r for r, _ in layers))
        from .rules import n_iterations, network_length_refined, network_length_uniform
        if d_max > d_min * (1 + 1e-9):
            nd = network_length_refined(eta, d_min, d_max, g, depth, zmax)
        else:
            nd = network_length_uniform(depth, d_min)
        out[k] = dict(depth=dd, growth=g, layers=layers, side=side, target=int(counts[rank]),
                      n_it=n_iterations(nd, 0.02))
    return out


def batch_bed(spec, seed, phi=0.636):
    """One bed of the batch grid on its square footprint, with bin walls and a
    0.1 m disc plate above the centre."""
    side = spec["side"]
    x, r = layered_bed(side, side, spec["layers"], spread=0.1, phi=phi, seed=seed)
    geoms = open_box_walls(side, side)
    zs = float((x[:, 2] + r).max())
    geoms.append(GeomSpec(CYLINDER, (side / 2, side / 2, zs + 0.005 + 0.001), he=(0.05, 0.0, 0.005),
                          mu_t=0.5, mu_r=0.02))
    mat = Material(rho=2600.0, mu_t=0.5, mu_r=0.02)
    return Bed(x, r, geoms, mat, name=f"batch bed depth {spec['depth']} growth {spec['growth']}",
               plate=len(geoms) - 1, plate_parts=(len(geoms) - 1,), box=(side, side, 0.25))


def refined_sinkage_bed(lx=0.89, ly=0.89, depth=0.25, seed=2503, phi=0.636):
    """Refined bed for plate sinkage: r = 2.5 mm in the top 2 cm, doubling per
    layer below (5, 10, 20 mm; max size ratio 8), 10% radius spread.  A
    0.89 x 0.89 m footprint gives about 200k spheres (the 0.4 x 0.4 m bin of
    the same layering holds about 41k).  A rigid disc plate (0.1 m diameter)
    above the centre is the driven geometry."""
    layers = refined_layers(depth=depth)
    x, r = layered_bed(lx, ly, layers, spread=0.1, phi=phi, seed=seed)
    geoms = open_box_walls(lx, ly)
    zs = float((x[:, 2] + r).max())
    plate = GeomSpec(CYLINDER, (lx / 2, ly / 2, zs + 0.01 + 0.005), he=(0.05, 0.0, 0.005),
                     mu_t=0.5, mu_r=0.02)
    geoms.append(plate)
    mat = Material(rho=2600.0, mu_t=0.5, mu_r=0.02)
    return Bed(x, r, geoms, mat, name=f"refined bed {lx}x{ly}x{depth} m, r 2.5/5/10/20 mm",
               plate=len(geoms) - 1, plate_parts=(len(geoms) - 1,), box=(lx, ly, depth))


def fine_shear_bed(lx=1.0, ly=0.5, depth=0.25, seed=2504, phi=0.636, r_nom=2.5e-3):
    """Homogeneous fine bed (r = 2.5 mm, 10% spread) with a 0.3 x 0.3 m plate
    carrying three transverse grousers 43 mm deep and 25.5 mm long at the
    bottom (Sec. 3.3); the plate and grousers are separate boxes."""
    x, r = layered_bed(lx, ly, [(r_nom, depth)], spread=0.1, phi=phi, seed=seed)
    geoms = open_box_walls(lx, ly)
    zs = float((x[:, 2] + r).max())
    cx, cy = 0.25 * lx, ly / 2
    t_plate = 0.01
    z_plate = zs + 0.043 + 0.002 + t_plate / 2
    parts = [GeomSpec(BOX, (cx, cy, z_plate), he=(0.15, 0.15, t_plate / 2), mu_t=0.5, mu_r=0.02)]
    for gx in (-0.1, 0.0, 0.1):
        parts.append(GeomSpec(BOX, (cx + gx, cy, z_plate - t_plate / 2 - 0.0215),
                              he=(0.01275, 0.15, 0.0215), mu_t=0.5, mu_r=0.02))
    first = len(geoms)
    geoms.extend(parts)
    mat = Material(rho=2600.0, mu_t=0.5, mu_r=0.02)
    return Bed(x, r, geoms, mat, name=f"fine bed {lx}x{ly}x{depth} m, r 2.5 mm",
               plate=first, plate_parts=tuple(range(first, len(geoms))), box=(lx, ly, depth))


SLICE = dict(lx=1.5, ly=0.17, depth=0.6)        # the shear-test container (Sec. 3.3)
H_GROUSER, L_GROUSER = 0.043, 0.0255             # grouser depth and length at the bottom (Sec. 3.3)


def shear_slice(d_min=8.5e-3, d_max=None, growth=1.25, eta=2.0, seed=2507, phi=0.636, plate_x=0.3,
                t_plate=0.01, n_grousers=3):
    """The pressure-sinkage / shear-displacement container of Sec. 3.3: a
    1.5 m long, 0.17 m wide slice of a bed 0.6 m deep, frictionless walls.
    Uniform particles of diameter d_min (d_max None), or refined: layers from
    the surface down with d_n = growth d_{n-1} and thickness eta d_n (Sec. 2.1),
    capped at d_max, which fills the rest (10% size spread in every layer).
    The plate is 0.3 m long and 0.5 m wide (wider than the slice), with
    n_grousers transverse grousers 43 mm deep and 25.5 mm long at the bottom;
    it starts clear above the particles (placed by the caller).  Material of
    Sec. 3.1 (dry sand: 2200 kg/m^3, E 1 GPa, nu 0.15, mu_t 0.3, mu_r 0.02);
    the plate takes the interparticle coefficients (Sec. 3.3)."""
    lx, ly, depth = SLICE["lx"], SLICE["ly"], SLICE["depth"]
    if d_max is None or d_max <= d_min:
        layers = [(d_min / 2, depth)]
        name = f"shear slice, uniform d {d_min * 1e3:.1f} mm"
    else:
        layers = graded_layers(d_min / 2, eta * d_min, growth, cap_ratio=d_max / d_min, depth=depth)
        name = (f"shear slice, refined d {d_min * 1e3:.1f} -> {d_max * 1e3:.1f} mm, growth {growth}, eta {eta}, "
                f"gamma {(growth - 1) / (growth * eta):.3f}")
    x, r = layered_bed(lx, ly, layers, spread=0.1, phi=phi, seed=seed)
    geoms = open_box_walls(lx, ly)
    cx, cy, z_plate = plate_x, ly / 2, depth + 1.0
    mat = Material(rho=RHO_PAPER, mu_t=MU_T_PAPER, mu_r=MU_R_PAPER)
    parts = [GeomSpec(BOX, (cx, cy, z_plate), he=(0.15, 0.25, t_plate / 2), mu_t=mat.mu_t, mu_r=mat.mu_r)]
    offs = np.linspace(-0.15 + L_GROUSER / 2, 0.15 - L_GROUSER / 2, n_grousers) if n_grousers > 1 else [0.0]
    for gx in offs:
        parts.append(GeomSpec(BOX, (cx + float(gx), cy, z_plate - t_plate / 2 - H_GROUSER / 2),
                              he=(L_GROUSER / 2, 0.25, H_GROUSER / 2), mu_t=mat.mu_t, mu_r=mat.mu_r))
    first = len(geoms)
    geoms.extend(parts)
    return Bed(x, r, geoms, mat, name=name, plate=first, plate_parts=tuple(range(first, len(geoms))),
               box=(lx, ly, depth))


def radial_zones(d_min, growth, eta, d_max, extent):
    """Zones (inner, outer distance, diameter) of a radially refined bed: zone n
    holds diameter d_n = d_min growth^n (capped at d_max) in a shell eta d_n
    thick, the layer rule of Sec. 2.1 applied to the distance from a point or
    an axis instead of the depth (the hemispheric and radial zones Sec. 5
    proposes); the capped size fills the rest out to `extent`."""
    zones, rho, d = [], 0.0, d_min
    while rho < extent:
        if d >= d_max * (1 - 1e-9):
            zones.append((rho, extent, d_max))
            break
        zones.append((rho, min(rho + eta * d, extent), d))
        rho += eta * d
        d = min(d * growth, d_max)
    return zones


def radially_refined_bed(lx=0.4, ly=0.4, depth=0.2, d_min=5e-3, growth=1.5, eta=3.0, d_max=20e-3,
                         centre=None, mode="hemisphere", spread=0.1, seed=2508, gap=0.03):
    """A bed refined around a point of its surface (mode "hemisphere": size
    grows with the distance from the point, hemispheric zones) or around a
    vertical axis through it (mode "cylinder": size grows with the horizontal
    distance, radial zones), zones from radial_zones.  Each zone is a jittered
    FCC lattice of its own size clipped to the zone, one radius (plus the
    jitter) inside each zone boundary, so no two spheres overlap; it settles
    under gravity like the layered beds.  Open box, frictionless walls."""
    rng = np.random.default_rng(seed)
    cx, cy = (lx / 2, ly / 2) if centre is None else centre
    extent = math.sqrt(max(cx, lx - cx) ** 2 + max(cy, ly - cy) ** 2 + (depth ** 2 if mode == "hemisphere" else 0.0))
    xs, rs = [], []
    for lo, hi, d in radial_zones(d_min, growth, eta, d_max, extent):
        r_nom = d / 2
        rmax = r_nom * (1 + spread)
        a = 2 * rmax * (1 + gap)
        jit = 0.45 * (a - 2 * rmax)
        m = rmax * 1.001 + jit
        # an FCC lattice over the box, then the zone's points
        dy, dz = a * math.sqrt(3.0) / 2.0, a * math.sqrt(2.0 / 3.0)
        pts = []
        for k in range(int((depth - 2 * m) / dz) + 1):
            sx, sy = (k % 3) * a / 2.0, (k % 3) * a * math.sqrt(3.0) / 6.0
            for j, y in enumerate(np.arange(m + sy, ly - m + 1e-12, dy)):
                xr = np.arange(m + sx + (a / 2.0 if j % 2 else 0.0), lx - m + 1e-12, a)
                pts.append(np.stack([xr, np.full_like(xr, y), np.full_like(xr, m + k * dz)], 1))
        p = np.concatenate(pts) if pts else np.zeros((0, 3))
        p = p + rng.uniform(-jit, jit, p.shape)
        # distance from the point at the surface (or from the axis)
        dh = np.hypot(p[:, 0] - cx, p[:, 1] - cy)
        dist = np.hypot(dh, depth - p[:, 2]) if mode == "hemisphere" else dh
        keep = (dist >= lo + m) & (dist <= hi - m) if lo > 0 else (dist <= hi - m)
        if hi >= extent:
            keep = dist >= lo + m
        p = p[keep]
        xs.append(p.astype(np.float64))
        rs.append(_uniform_radii(rng, r_nom, len(p), spread))
    x, r = np.concatenate(xs), np.concatenate(rs)
    mat = Material(rho=RHO_PAPER, mu_t=MU_T_PAPER, mu_r=MU_R_PAPER)
    return Bed(x, r, open_box_walls(lx, ly), mat, box=(lx, ly, depth),
               name=f"{mode} refined bed d {d_min * 1e3:.1f} -> {d_max * 1e3:.1f} mm, growth {growth}, eta {eta}")


def shear_slice_layers(d_min, d_max, growth, eta, depth=0.6):
    """(layers bottom up, refined depth z_max) of shear_slice's refined bed, for Eq. 10."""
    layers = graded_layers(d_min / 2, eta * d_min, growth, cap_ratio=d_max / d_min, depth=depth)
    zmax = sum(t for r, t in layers[1:])
    return layers, zmax


def random_cloud(n, seed, rmin=2e-3, rmax=6e-3, box=0.05, overlap_ok=False, vscale=0.0):
    """Spheres placed uniformly at random in [-box, box]^3 (overlaps allowed
    unless overlap_ok is False, then rejection sampled); velocities uniform in
    [-vscale, vscale]."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(rmin, rmax, n).astype(np.float32)
    if overlap_ok:
        x = rng.uniform(-box, box, (n, 3))
    else:
        x = np.zeros((n, 3))
        for i in range(n):
            for _ in range(10000):
                c = rng.uniform(-box, box, 3)
                if i == 0 or (np.linalg.norm(x[:i] - c, axis=1) > r[:i].astype(float) + float(r[i])).all():
                    break
            x[i] = c
    v = rng.uniform(-vscale, vscale, (n, 3)).astype(np.float32)
    w = rng.uniform(-vscale, vscale, (n, 3)).astype(np.float32) * 100.0
    return x.astype(np.float64), r, v, w


def column(n, r=5e-3):
    """n equal spheres stacked on the floor plane, just touching."""
    x = np.array([[0.0, 0.0, r + 2 * r * k] for k in range(n)])
    return x, np.full(n, r, np.float32)


# triaxial cell: wall indices of cell_walls()
FLOOR, PLATEN, WALL_XLO, WALL_XHI, WALL_YLO, WALL_YHI = range(6)


def cell_walls(lo, hi, v_top=0.0, mu_wall=0.0):
    """The six walls of a box-shaped triaxial cell around [lo, hi]: floor, top
    platen moving with velocity (0, 0, v_top), and four side walls.  Wall
    friction and rolling resistance are zero in the paper's triaxial tests
    (Sec. 3.2)."""
    walls = [plane((0, 0, lo[2]), (0, 0, 1), mu_wall, mu_wall),
             plane((0, 0, hi[2]), (0, 0, -1), mu_wall, mu_wall),
             plane((lo[0], 0, 0), (1, 0, 0), mu_wall, mu_wall),
             plane((hi[0], 0, 0), (-1, 0, 0), mu_wall, mu_wall),
             plane((0, lo[1], 0), (0, 1, 0), mu_wall, mu_wall),
             plane((0, hi[1], 0), (0, -1, 0), mu_wall, mu_wall)]
    walls[PLATEN] = replace(walls[PLATEN], v=(0.0, 0.0, float(v_top)))
    return walls


def triaxial_cell(n=50_000, rmin=2.5e-3, rmax=3.0e-3, seed=2505, gap=0.01, squeeze=0.0, v_top=0.0):
    """n spheres, r ~ U[rmin, rmax], on a jittered FCC lattice filling a cube,
    inside the six walls of a box triaxial cell (Sec. 3.2).  `squeeze` > 0
    scales the lattice about its centre by (1 - squeeze) so that neighbours
    overlap, and moves every wall into the outermost spheres by squeeze * rmin:
    a pre-stressed sample without a consolidation run."""
    rng = np.random.default_rng(seed)
    r_nom, spread = 0.5 * (rmin + rmax), (rmax - rmin) / (rmin + rmax)
    a = 2 * rmax * (1 + gap)
    side = a * (n / math.sqrt(2.0)) ** (1.0 / 3.0) + 2.0 * rmax
    for _ in range(6):   # footprint whose stack height matches it
        x, r, ztop = lattice_layer(np.random.default_rng(seed), side, side, 0.0, n, r_nom, spread, gap)
        side *= (ztop / side) ** (1.0 / 3.0)
    x, r, ztop = lattice_layer(rng, side, side, 0.0, n, r_nom, spread, gap)
    if squeeze > 0:
        c = 0.5 * (x.min(0) + x.max(0))
        x = c + (x - c) * (1.0 - squeeze)
    rr = r.astype(np.float64)[:, None]
    inset = squeeze * rmin
    lo = (x - rr).min(0) + inset
    hi = (x + rr).max(0) - inset
    mat = Material(rho=2600.0, mu_t=0.5, mu_r=0.02)
    return Bed(x, r, cell_walls(lo, hi, v_top), mat, plate=PLATEN,
               name=f"triaxial cell, {n} spheres r~U[{rmin * 1e3:g},{rmax * 1e3:g}] mm",
               box=tuple(map(float, hi - lo)))


def triaxial_refined_cell(side=0.2, r_fine=2.75e-3, growth=2.0, seed=2506, gap=0.01):
    """A triaxial cell of the fine cell's size whose lower half holds spheres
    `growth` times larger (10% spread): a two-layer refined sample (Sec. 2.1)
    inside the six walls of a box cell (Sec. 3.2)."""
    x, r = layered_bed(side, side, [(r_fine * growth, side / 2), (r_fine, side / 2)], spread=0.1, seed=seed,
                       gap=gap)
    rr = r.astype(np.float64)[:, None]
    lo, hi = (x - rr).min(0), (x + rr).max(0)
    mat = Material(rho=2600.0, mu_t=0.5, mu_r=0.02)
    return Bed(x, r, cell_walls(lo, hi), mat, plate=PLATEN,
               name=f"refined triaxial cell, {len(r)} spheres r {r_fine * 1e3:g}/{r_fine * growth * 1e3:g} mm",
               box=tuple(map(float, hi - lo)))
