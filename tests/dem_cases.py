"""Shared set-up of GPU-vs-oracle comparisons: one bed, two implementations.

Both sides receive the same seeded inputs (positions as float64, radii and
velocities rounded to float32, every material and solver constant rounded to
float32), so the only differences are the GPU's FP32 arithmetic and summation
order.  Nothing here computes any part of the method.
"""
import numpy as np

import oracle
from oracle import Geom, OracleParams
from paper_2501_05300_gb300 import beds


def f32(x):
    return float(np.float32(x))


PARAMS = dict(rho=2600.0, E=1e9, nu=0.15, mu_t=0.5, mu_r=0.02, e_H=1.25, damp_steps=4.5,
              dt=1e-5, n_it=100, gravity=(0.0, 0.0, -9.81), kn_scale=1.0, eps_reg=1e-6,
              delta_floor=1e-8)


def params(**over):
    p = dict(PARAMS)
    p.update(over)
    for k, v in list(p.items()):
        if k == "n_it":
            continue
        p[k] = tuple(f32(x) for x in v) if isinstance(v, tuple) else f32(v)
    return p


def oracle_geoms(geoms):
    return [Geom(g.type, tuple(g.c), tuple(g.R), tuple(g.he), tuple(g.v), tuple(g.w),
                 f32(g.E), f32(g.nu), f32(g.mu_t), f32(g.mu_r)) for g in geoms]


def make_oracle(x, r, p, geoms=(), v=None, w=None):
    op = OracleParams(**p)
    v = None if v is None else np.asarray(v, np.float32).astype(np.float64)
    w = None if w is None else np.asarray(w, np.float32).astype(np.float64)
    return oracle.Oracle(op, x, np.asarray(r, np.float32).astype(np.float64), v, w,
                         geoms=oracle_geoms(geoms))


def make_gpu(x, r, p, geoms=(), v=None, w=None, **kw):
    from paper_2501_05300_gb300.dem import Bed
    if not hasattr(r, "data_ptr"):
        r = np.asarray(r, np.float32)
    return Bed(x, r, v=v, w=w, geoms=geoms, **p, **kw)


def canonical_gpu_contacts(a, b, lam):
    """Re-orient GPU contacts like the oracle: body a = lower stable id."""
    a = a.astype(np.int64).copy(); b = b.astype(np.int64).copy()
    lam = lam.astype(np.float64).copy()
    flip = (b >= 0) & (a > b)
    a[flip], b[flip] = b[flip], a[flip].copy()
    lam[flip, 1:] *= -1.0
    order = np.lexsort((b, a))
    return a[order], b[order], lam[order], order


def compressed_cloud(n, seed, rmin=2.5e-3, rmax=5.5e-3, box=None, squeeze=0.92):
    """Spheres on a jittered cubic lattice whose spacing is shrunk below the
    mean diameter, so that many neighbours overlap (a dense contact network
    without settling); radii span several grid levels."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(rmin, rmax, n).astype(np.float32)
    s = squeeze * (rmin + rmax)
    k = int(np.ceil(n ** (1 / 3)))
    idx = np.arange(n)
    g = np.stack([idx % k, (idx // k) % k, idx // (k * k)], 1).astype(np.float64)
    x = g * s + rng.uniform(-0.1, 0.1, (n, 3)) * s + rmax
    return x, r


def box_geoms(lo, hi, mu=0.3):
    """Floor and four walls around [lo, hi] (frictional) plus nothing else."""
    gs = [beds.plane((0, 0, lo[2]), (0, 0, 1), mu, 0.01),
          beds.plane((lo[0], 0, 0), (1, 0, 0), mu, 0.01),
          beds.plane((hi[0], 0, 0), (-1, 0, 0), mu, 0.01),
          beds.plane((0, lo[1], 0), (0, 1, 0), mu, 0.01),
          beds.plane((0, hi[1], 0), (0, -1, 0), mu, 0.01)]
    for g in gs:
        g.mu_t, g.mu_r = mu, 0.01
    return gs


def primitive_cloud(n=150, seed=7):
    """A compressed cloud in a frictional box, pressed by an oblique box
    (translating down and sideways) and a tilted cylinder (translating): the
    contacts include box faces, edges and corners, and cylinder caps, sides
    and rims.  Primitives 5 (box) and 6 (cylinder) follow the five walls."""
    from scipy.spatial.transform import Rotation
    x, r = compressed_cloud(n, seed=seed)
    lo, hi = x.min(0) - 0.004, x.max(0) + 0.004
    geoms = box_geoms(lo, hi)
    c = (lo + hi) / 2
    Rb = Rotation.from_euler("xyz", [0.3, -0.2, 0.5]).as_matrix().reshape(-1)
    Rc = Rotation.from_euler("xyz", [0.6, 0.4, 0.0]).as_matrix().reshape(-1)
    geoms.append(beds.GeomSpec(beds.BOX, (c[0], c[1], hi[2] - 0.004), tuple(Rb), (0.012, 0.008, 0.005),
                               v=(0.01, 0.0, -0.05), mu_t=0.4, mu_r=0.02))
    geoms.append(beds.GeomSpec(beds.CYLINDER, (lo[0] + 0.01, lo[1] + 0.01, c[2]), tuple(Rc),
                               he=(0.007, 0.0, 0.006), v=(0.0, 0.02, 0.0), mu_t=0.4, mu_r=0.02))
    return x, r, geoms
