"""ctypes binding of libdem.so (include/dem.h).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  The module-level functions carry the C names; `Bed` wraps them for
convenience.  Device memory for a bed comes from PyTorch's caching allocator
(through the allocator hooks of dem_bed_desc) and the bed runs on a PyTorch
CUDA stream.  If the library cannot be loaded an ImportError is raised: there
is no CPU fallback.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref

import numpy as np

from . import buildlib as _build

DEM_OK, DEM_ERR_ARG, DEM_ERR_CUDA, DEM_ERR_CAPACITY, DEM_ERR_TIMEOUT, DEM_ERR_NONFINITE, DEM_ERR_STATE = range(7)
STATUS = {0: "DEM_OK", 1: "DEM_ERR_ARG", 2: "DEM_ERR_CUDA", 3: "DEM_ERR_CAPACITY",
          4: "DEM_ERR_TIMEOUT", 5: "DEM_ERR_NONFINITE", 6: "DEM_ERR_STATE"}
PLANE, BOX, CYLINDER = 0, 1, 2

# every entry point declared in include/dem.h
EXPORTS = ("dem_create_bed", "dem_create_batch", "dem_autotune", "dem_step", "dem_apply_plate_velocity", "dem_read_forces",
           "dem_read_state", "dem_read_contacts", "dem_read_geom", "dem_sync", "dem_get_info",
           "dem_set_timing", "dem_read_timing", "dem_set_params", "dem_apply_plate_load", "dem_set_plate_load",
           "dem_record", "dem_step_adjoint",
           "dem_checkpoint_save", "dem_checkpoint_restore", "dem_checkpoint_free",
           "dem_destroy_bed", "dem_detect_contacts_noalloc", "dem_last_error")


class DemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class dem_geom(C.Structure):
    _fields_ = [("type", C.c_int32), ("c", C.c_double * 3), ("R", C.c_double * 9),
                ("he", C.c_double * 3), ("v", C.c_double * 3), ("w", C.c_double * 3),
                ("E", C.c_float), ("nu", C.c_float), ("mu_t", C.c_float), ("mu_r", C.c_float)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class dem_bed_desc(C.Structure):
    _fields_ = [("n", C.c_int32), ("pos", C.c_void_p), ("radius", C.c_void_p), ("vel", C.c_void_p),
                ("omega", C.c_void_p), ("inv_mass", C.c_void_p), ("inv_inertia", C.c_void_p),
                ("rho", C.c_float), ("E", C.c_float), ("nu", C.c_float), ("mu_t", C.c_float),
                ("mu_r", C.c_float), ("e_H", C.c_float), ("damp_steps", C.c_float), ("dt", C.c_float),
                ("n_it", C.c_int32), ("gravity", C.c_float * 3), ("kn_scale", C.c_float),
                ("eps_reg", C.c_float), ("delta_floor", C.c_float), ("n_geom", C.c_int32),
                ("geom", C.POINTER(dem_geom)), ("contact_capacity", C.c_int64),
                ("resort_every", C.c_int32), ("level_ratio", C.c_float), ("lanes", C.c_int32),
                ("alloc", ALLOC_FN),
                ("free_fn", FREE_FN), ("alloc_ctx", C.c_void_p), ("solver", C.c_int32),
                ("restitution", C.c_float), ("impact_speed", C.c_float)]


class dem_info(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_levels", C.c_int32), ("n_cells", C.c_int64),
                ("contacts", C.c_int64), ("geom_contacts", C.c_int64), ("steps", C.c_int64),
                ("contact_capacity", C.c_int64), ("kernels_per_step", C.c_int32),
                ("kernels_per_resort", C.c_int32), ("n_beds", C.c_int32), ("lanes", C.c_int32),
                ("resort_every", C.c_int32), ("solver", C.c_int32), ("colours", C.c_int32),
                ("impacts", C.c_int64)]


_lib = None
_live = weakref.WeakSet()   # open beds, closed before the interpreter (and torch) shut down


@atexit.register
def _close_all():
    for b in list(_live):
        try:
            b.close()
        except Exception:
            pass


def lib_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load libdem.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"{_build.LIB} is missing: build the CUDA library first")
    lib = C.CDLL(_build.LIB)
    vp, i32, i64, dp, fp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double), C.c_void_p
    sigs = {
        "dem_create_bed": (i32, [C.POINTER(dem_bed_desc), vp, C.POINTER(vp)]),
        "dem_create_batch": (i32, [C.POINTER(dem_bed_desc), i32, vp, C.POINTER(vp)]),
        "dem_autotune": (i32, [vp, i32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "dem_step": (i32, [vp, i32]),
        "dem_apply_plate_velocity": (i32, [vp, i32, dp, dp]),
        "dem_read_forces": (i32, [vp, i32, dp, dp, dp]),
        "dem_read_state": (i32, [vp, vp, vp, vp, i32]),
        "dem_read_contacts": (i32, [vp, i64, vp, vp, vp, vp, C.POINTER(C.c_int64)]),
        "dem_read_geom": (i32, [vp, i32, C.POINTER(dem_geom)]),
        "dem_sync": (i32, [vp]),
        "dem_get_info": (i32, [vp, C.POINTER(dem_info)]),
        "dem_set_timing": (i32, [vp, i32]),
        "dem_read_timing": (i32, [vp, dp, dp, C.POINTER(C.c_int64)]),
        "dem_set_params": (i32, [vp, C.POINTER(dem_bed_desc)]),
        "dem_apply_plate_load": (i32, [vp, vp, i32, C.c_double, dp, i32]),
        "dem_set_plate_load": (i32, [vp, i32, dp]),
        "dem_record": (i32, [vp, i32, i32, vp]),
        "dem_step_adjoint": (i32, [vp, vp, dp]),
        "dem_checkpoint_save": (i32, [vp, C.POINTER(vp)]),
        "dem_checkpoint_restore": (i32, [vp, vp]),
        "dem_checkpoint_free": (i32, [vp, vp]),
        "dem_destroy_bed": (i32, [vp]),
        "dem_detect_contacts_noalloc": (i32, [i32, vp, vp, i64, vp, vp, vp, vp, vp]),
        "dem_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().dem_last_error().decode()


def _check(st):
    if st != DEM_OK:
        raise DemError(st, last_error())


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _input(a, dtype, shape):
    """An input array as numpy (host) or as a contiguous torch tensor of the
    right dtype (host or device memory; the library reads either)."""
    if hasattr(a, "data_ptr"):
        import torch
        td = torch.float64 if dtype == np.float64 else torch.float32
        return a.detach().to(dtype=td).contiguous().reshape(shape)
    return np.ascontiguousarray(a, dtype=dtype).reshape(shape)


def geom_struct(g) -> dem_geom:
    """A dem_geom from any object with the GeomSpec fields."""
    s = dem_geom()
    s.type = int(g.type)
    s.c = (C.c_double * 3)(*map(float, g.c))
    s.R = (C.c_double * 9)(*map(float, g.R))
    s.he = (C.c_double * 3)(*map(float, g.he))
    s.v = (C.c_double * 3)(*map(float, g.v))
    s.w = (C.c_double * 3)(*map(float, g.w))
    s.E, s.nu, s.mu_t, s.mu_r = float(g.E), float(g.nu), float(g.mu_t), float(g.mu_r)
    return s


class _TorchAllocator:
    """Allocator hooks that take device memory from PyTorch's caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx, stream):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0)
        except Exception:
            return None

    def _free(self, ptr, ctx, stream):
        self.torch.cuda.caching_allocator_delete(ptr)


def _make_desc(x, r, keep, *, v=None, w=None, geoms=(), rho=2600.0, E=1e9, nu=0.15, mu_t=0.5,
               mu_r=0.02, e_H=1.25, damp_steps=4.5, dt=1e-5, n_it=100, gravity=(0.0, 0.0, -9.81),
               kn_scale=1.0, eps_reg=1e-6, delta_floor=0.0, inv_mass=None, inv_inertia=None,
               contact_capacity=0, resort_every=0, level_ratio=0.0, lanes=0, solver=0, restitution=0.0,
               impact_speed=0.0):
    """A dem_bed_desc for one bed; arrays that must outlive the call go to keep."""
    x = _input(x, np.float64, (-1, 3))
    r = _input(r, np.float32, (-1,))
    n = int(r.shape[0])
    if int(x.shape[0]) != n:
        raise ValueError("x and r disagree in length")
    keep += [x, r]
    d = dem_bed_desc()
    d.n = n
    d.pos, d.radius = _ptr(x), _ptr(r)
    for name, arr, shape in (("vel", v, (n, 3)), ("omega", w, (n, 3)), ("inv_mass", inv_mass, (n,)),
                             ("inv_inertia", inv_inertia, (n,))):
        if arr is not None:
            a = _input(arr, np.float32, shape)
            keep.append(a)
            setattr(d, name, _ptr(a))
    d.rho, d.E, d.nu, d.mu_t, d.mu_r = rho, E, nu, mu_t, mu_r
    d.e_H, d.damp_steps, d.dt, d.n_it = e_H, damp_steps, dt, int(n_it)
    d.gravity = (C.c_float * 3)(*map(float, gravity))
    d.kn_scale, d.eps_reg, d.delta_floor = kn_scale, eps_reg, delta_floor
    geoms = list(geoms)
    garr = (dem_geom * max(1, len(geoms)))(*[geom_struct(g) for g in geoms])
    keep.append(garr)
    d.n_geom = len(geoms)
    d.geom = C.cast(garr, C.POINTER(dem_geom))
    d.contact_capacity = int(contact_capacity)
    d.resort_every = int(resort_every)
    d.level_ratio = float(level_ratio)
    d.lanes = int(lanes)
    d.solver = int(solver)
    d.restitution, d.impact_speed = float(restitution), float(impact_speed)
    return d, n, geoms


_SOLVER_KEYS = dict(dt=1e-5, n_it=100, mu_t=0.5, mu_r=0.02, damp_steps=4.5, e_H=1.25,
                    gravity=(0.0, 0.0, -9.81), kn_scale=1.0, eps_reg=1e-6)


def _solver_params(kw):
    return {k: kw.get(k, v) for k, v in _SOLVER_KEYS.items()}


class Bed:
    """A bed of spheres advanced by the CUDA library.

    x: float64 [N,3] centres, r: float32 [N] radii, geoms: objects with the
    GeomSpec fields.  Material and solver parameters follow dem_bed_desc."""

    def __init__(self, x, r, *, stream=None, use_torch=True, **kw):
        self.lib = load()
        self._handle = C.c_void_p()
        keep = []
        d, n, geoms = _make_desc(x, r, keep, **kw)
        self.geoms = geoms
        self.n = n
        self.dt = kw.get("dt", 1e-5)
        self.params = _solver_params(kw)
        self._create([d], keep, stream, use_torch)

    def _create(self, descs, keep, stream, use_torch):
        self._alloc = None
        self._ckpts = []
        stream_ptr = None
        if use_torch:
            import torch
            self._alloc = _TorchAllocator(torch.cuda.current_device())
            if stream is None:
                stream = torch.cuda.current_stream()
        if stream is not None:
            # a handle of 0 (the legacy default stream) makes the library use a stream of its own
            stream_ptr = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        arr = (dem_bed_desc * len(descs))(*descs)
        for d in arr:
            if self._alloc is not None:
                d.alloc, d.free_fn = self._alloc.alloc, self._alloc.free
        self.stream = stream
        if len(descs) == 1:
            _check(self.lib.dem_create_bed(C.cast(arr, C.POINTER(dem_bed_desc)), stream_ptr, C.byref(self._handle)))
        else:
            _check(self.lib.dem_create_batch(C.cast(arr, C.POINTER(dem_bed_desc)), len(descs), stream_ptr,
                                             C.byref(self._handle)))
        _live.add(self)

    # -- the C entry points -------------------------------------------------
    def step(self, nsteps=1):
        _check(self.lib.dem_step(self._handle, int(nsteps)))

    def autotune(self, trial_steps=5):
        """Pick the sweep layout and re-sort period by timing (dem_autotune)."""
        a, b = C.c_int32(), C.c_int32()
        _check(self.lib.dem_autotune(self._handle, int(trial_steps), C.byref(a), C.byref(b)))
        return a.value, b.value

    def apply_plate_velocity(self, g, v, w=(0.0, 0.0, 0.0)):
        vv = (C.c_double * 3)(*map(float, v))
        ww = (C.c_double * 3)(*map(float, w))
        _check(self.lib.dem_apply_plate_velocity(self._handle, int(g), vv, ww))

    def apply_plate_load(self, geoms, mass, force, dof=4):
        """Make the primitives one load-driven rigid group (dem_apply_plate_load)."""
        g = np.ascontiguousarray(np.atleast_1d(geoms), np.int32)
        f = (C.c_double * 3)(*map(float, force))
        _check(self.lib.dem_apply_plate_load(self._handle, _ptr(g), len(g), float(mass), f, int(dof)))

    def set_plate_load(self, g, force):
        """New external force [N] of the load-driven group holding primitive g
        (dem_set_plate_load), from the next step on."""
        f = (C.c_double * 3)(*map(float, force))
        _check(self.lib.dem_set_plate_load(self._handle, int(g), f))

    def read_forces(self, g):
        f = (C.c_double * 3)()
        t = (C.c_double * 3)()
        s = C.c_double()
        _check(self.lib.dem_read_forces(self._handle, int(g), f, t, C.byref(s)))
        return np.array(f[:]), np.array(t[:]), s.value

    def read_state(self):
        x = np.zeros((self.n, 3), np.float64)
        v = np.zeros((self.n, 3), np.float32)
        w = np.zeros((self.n, 3), np.float32)
        _check(self.lib.dem_read_state(self._handle, _ptr(x), _ptr(v), _ptr(w), self.n))
        return x, v, w

    def read_contacts(self):
        """(key_a, key_b, lam7, delta) of the last step."""
        cnt = C.c_int64()
        _check(self.lib.dem_read_contacts(self._handle, 0, None, None, None, None, C.byref(cnt)))
        m = cnt.value
        a = np.zeros(m, np.int32); b = np.zeros(m, np.int32)
        lam = np.zeros((m, 7), np.float32); dl = np.zeros(m, np.float32)
        _check(self.lib.dem_read_contacts(self._handle, m, _ptr(a), _ptr(b), _ptr(lam), _ptr(dl),
                                          C.byref(cnt)))
        return a, b, lam, dl

    def read_geom(self, g):
        out = dem_geom()
        _check(self.lib.dem_read_geom(self._handle, int(g), C.byref(out)))
        return out

    def sync(self):
        _check(self.lib.dem_sync(self._handle))

    def info(self) -> dem_info:
        out = dem_info()
        _check(self.lib.dem_get_info(self._handle, C.byref(out)))
        return out

    def set_timing(self, enable=True):
        _check(self.lib.dem_set_timing(self._handle, 1 if enable else 0))

    def read_timing(self):
        a, j, s = C.c_double(), C.c_double(), C.c_int64()
        _check(self.lib.dem_read_timing(self._handle, C.byref(a), C.byref(j), C.byref(s)))
        return a.value, j.value, s.value

    def set_params(self, *, dt, n_it, mu_t, mu_r, damp_steps=4.5, e_H=1.25, gravity=(0.0, 0.0, -9.81),
                   kn_scale=1.0, eps_reg=1e-6, lanes=0, solver=-1, restitution=-1.0, impact_speed=-1.0):
        """Change solver and material settings between steps (dem_set_params);
        solver, restitution and impact_speed -1 keep the current ones."""
        d = dem_bed_desc()
        d.dt, d.n_it, d.mu_t, d.mu_r, d.damp_steps, d.e_H = dt, int(n_it), mu_t, mu_r, damp_steps, e_H
        d.gravity = (C.c_float * 3)(*map(float, gravity))
        d.kn_scale, d.eps_reg, d.lanes, d.solver = kn_scale, eps_reg, int(lanes), int(solver)
        d.restitution, d.impact_speed = float(restitution), float(impact_speed)
        _check(self.lib.dem_set_params(self._handle, C.byref(d)))
        self.dt = dt
        self.params = dict(dt=dt, n_it=int(n_it), mu_t=mu_t, mu_r=mu_r, damp_steps=damp_steps, e_H=e_H,
                           gravity=tuple(gravity), kn_scale=kn_scale, eps_reg=eps_reg)

    def set_material(self, *, kn_scale=None, mu_t=None, mu_r=None):
        """Change the stiffness scale and the friction coefficients only; the
        sweep layout is kept."""
        p = dict(self.params)
        for k, v in (("kn_scale", kn_scale), ("mu_t", mu_t), ("mu_r", mu_r)):
            if v is not None:
                p[k] = float(v)
        if all(p[k] == self.params[k] for k in ("kn_scale", "mu_t", "mu_r")):
            return
        self.set_params(**p, lanes=-1)

    def record(self, nsteps, ckpt_every=0):
        """Advance nsteps steps keeping checkpoints for the adjoint
        (dem_record).  Returns the force on every primitive in every step,
        shape (nsteps, n_geom, 3) [N]."""
        f = np.zeros((int(nsteps), len(self.geoms), 3), np.float64)
        _check(self.lib.dem_record(self._handle, int(nsteps), int(ckpt_every), _ptr(f)))
        return f

    def save_checkpoint(self):
        """A device copy of the bed's state (dem_checkpoint_save)."""
        h = C.c_void_p()
        _check(self.lib.dem_checkpoint_save(self._handle, C.byref(h)))
        self._ckpts.append(h)
        return h

    def restore_checkpoint(self, h):
        _check(self.lib.dem_checkpoint_restore(self._handle, h))

    def free_checkpoint(self, h):
        _check(self.lib.dem_checkpoint_free(self._handle, h))
        self._ckpts = [c for c in self._ckpts if c.value != h.value]

    def adjoint(self, dJ_dF):
        """dJ/d(kn_scale, mu_t, mu_r) of J = sum dJ_dF * F over the recorded
        window (dem_step_adjoint)."""
        w = _input(dJ_dF, np.float64, (-1, len(self.geoms), 3))
        g = (C.c_double * 3)()
        _check(self.lib.dem_step_adjoint(self._handle, _ptr(w), g))
        return np.array(g[:])

    def close(self):
        if getattr(self, "_handle", None) and self._handle.value:
            for h in getattr(self, "_ckpts", []):
                self.lib.dem_checkpoint_free(self._handle, h)
            self._ckpts = []
            self.lib.dem_destroy_bed(self._handle)
            self._handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch(Bed):
    """Several independent beds advanced together (dem_create_batch).

    beds: list of dicts with the keyword arguments of Bed (x, r, geoms, n_it,
    ...); shared settings must agree.  Particle and primitive numbers are
    global: bed k's come after those of beds 0..k-1 (see offsets)."""

    def __init__(self, beds, *, stream=None, use_torch=True, **shared):
        self.lib = load()
        self._handle = C.c_void_p()
        keep, descs = [], []
        self.offsets, self.geom_offsets = [], []
        n = ng = 0
        self.geoms = []
        for spec in beds:
            kw = dict(shared)
            kw.update({k: v for k, v in spec.items() if k not in ("x", "r")})
            d, m, geoms = _make_desc(spec["x"], spec["r"], keep, **kw)
            descs.append(d)
            self.offsets.append(n)
            self.geom_offsets.append(ng)
            self.geoms += geoms
            n += m
            ng += len(geoms)
        self.n = n
        self.dt = shared.get("dt", 1e-5)
        self.params = _solver_params(shared)
        self._create(descs, keep, stream, use_torch)


def detect_contacts_noalloc(pos, radius, key_a, key_b, delta, count, stream=None):
    """dem_detect_contacts_noalloc on torch CUDA tensors (pos float64 [n,3],
    radius float32 [n], outputs int32/int32/float32 [cap], count int64 [1]).
    The library allocates nothing; the caller owns every buffer."""
    lib = load()
    n = int(radius.shape[0])
    sp = None if stream is None else C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib.dem_detect_contacts_noalloc(n, _ptr(pos), _ptr(radius), int(key_a.shape[0]), _ptr(key_a),
                                           _ptr(key_b), _ptr(delta), _ptr(count), sp))


def bed_from(spec, *, n_it, dt, **kw) -> Bed:
    """A Bed from a beds.Bed description (positions, radii, geometry, material)."""
    m = spec.material
    kw.setdefault("rho", m.rho)
    kw.setdefault("E", m.E)
    kw.setdefault("nu", m.nu)
    kw.setdefault("mu_t", m.mu_t)
    kw.setdefault("mu_r", m.mu_r)
    return Bed(spec.x, spec.r, geoms=spec.geoms, n_it=n_it, dt=dt, **kw)
