"""ctypes binding of the FP64 oracle (oracle.c).  Test infrastructure only."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

PLANE, BOX, CYLINDER = 0, 1, 2


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile liboracle.so in place (gcc, OpenMP, no fused multiply-add)."""
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("rho", C.c_double), ("E", C.c_double), ("nu", C.c_double),
                ("mu_t", C.c_double), ("mu_r", C.c_double), ("e_H", C.c_double),
                ("damp_steps", C.c_double), ("dt", C.c_double), ("n_it", C.c_int32),
                ("gravity", C.c_double * 3), ("kn_scale", C.c_double),
                ("eps_reg", C.c_double), ("delta_floor", C.c_double), ("solver", C.c_int32),
                ("e_imp", C.c_double), ("v_imp", C.c_double)]


class _Geom(C.Structure):
    _fields_ = [("type", C.c_int32), ("c", C.c_double * 3), ("R", C.c_double * 9),
                ("he", C.c_double * 3), ("v", C.c_double * 3), ("w", C.c_double * 3),
                ("E", C.c_double), ("nu", C.c_double), ("mu_t", C.c_double),
                ("mu_r", C.c_double)]


@dataclass
class OracleParams:
    rho: float = 2600.0
    E: float = 1e9
    nu: float = 0.15
    mu_t: float = 0.5
    mu_r: float = 0.02
    e_H: float = 1.25
    damp_steps: float = 4.5
    dt: float = 1e-5
    n_it: int = 100
    gravity: tuple = (0.0, 0.0, -9.81)
    kn_scale: float = 1.0
    eps_reg: float = 1e-6
    delta_floor: float = 1e-8
    solver: int = 0              # 0 Jacobi with mass splitting, 1 coloured projected Gauss-Seidel
    restitution: float = 0.0     # Newton impact law: restitution coefficient (Sec. 2.2)
    impact_speed: float = 0.0    # impact threshold [m/s]; 0 = no impact stage

    def to_c(self) -> _Params:
        p = _Params()
        for k in ("rho", "E", "nu", "mu_t", "mu_r", "e_H", "damp_steps", "dt", "kn_scale",
                  "eps_reg", "delta_floor"):
            setattr(p, k, float(getattr(self, k)))
        p.n_it = int(self.n_it)
        p.solver = int(self.solver)
        p.e_imp = float(self.restitution)
        p.v_imp = float(self.impact_speed)
        p.gravity = (C.c_double * 3)(*[float(v) for v in self.gravity])
        return p


@dataclass
class Geom:
    type: int
    c: tuple
    R: tuple = (1, 0, 0, 0, 1, 0, 0, 0, 1)
    he: tuple = (0.0, 0.0, 0.0)
    v: tuple = (0.0, 0.0, 0.0)
    w: tuple = (0.0, 0.0, 0.0)
    E: float = 1e9
    nu: float = 0.15
    mu_t: float = 0.5
    mu_r: float = 0.02

    def to_c(self) -> _Geom:
        g = _Geom()
        g.type = int(self.type)
        g.c = (C.c_double * 3)(*map(float, self.c))
        g.R = (C.c_double * 9)(*map(float, self.R))
        g.he = (C.c_double * 3)(*map(float, self.he))
        g.v = (C.c_double * 3)(*map(float, self.v))
        g.w = (C.c_double * 3)(*map(float, self.w))
        g.E, g.nu, g.mu_t, g.mu_r = float(self.E), float(self.nu), float(self.mu_t), float(self.mu_r)
        return g

    @staticmethod
    def from_c(g: _Geom) -> "Geom":
        return Geom(g.type, tuple(g.c), tuple(g.R), tuple(g.he), tuple(g.v), tuple(g.w),
                    g.E, g.nu, g.mu_t, g.mu_r)


_lib = None


def load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = np.ctypeslib.ndpointer
        d = P(dtype=np.float64, flags="C_CONTIGUOUS")
        i32 = P(dtype=np.int32, flags="C_CONTIGUOUS")
        vp = C.c_void_p
        lib.orc_detect.restype = C.c_int64
        lib.orc_detect.argtypes = [C.c_int32, d, d, i32, C.c_int32, vp, C.c_int64, i32, i32, d]
        lib.orc_create.restype = vp
        lib.orc_create.argtypes = [C.POINTER(_Params), C.c_int32, d, d, d, d, i32, vp, vp,
                                   C.c_int32, vp]
        lib.orc_destroy.argtypes = [vp]
        lib.orc_step.argtypes = [vp, C.c_int32]
        lib.orc_get_state.argtypes = [vp, vp, vp, vp]
        lib.orc_set_state.argtypes = [vp, vp, vp, vp]
        lib.orc_set_geom_velocity.argtypes = [vp, C.c_int32, d, d]
        lib.orc_get_geom.argtypes = [vp, C.c_int32, C.POINTER(_Geom)]
        lib.orc_get_geom_force.argtypes = [vp, C.c_int32, d, d]
        lib.orc_get_contacts.restype = C.c_int64
        lib.orc_get_contacts.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp]
        lib.orc_set_warmstart.argtypes = [vp, C.c_int64, i32, i32, d]
        lib.orc_threads.restype = C.c_int
        lib.orc_colours.restype = C.c_int32
        lib.orc_colours.argtypes = [vp]
        lib.orc_impacts.restype = C.c_int64
        lib.orc_impacts.argtypes = [vp]
        lib.orc_step.restype = C.c_int
        lib.orc_set_load.restype = C.c_int
        lib.orc_set_load.argtypes = [vp, C.c_int32, i32, C.c_double, d, C.c_int32]
        lib.orc_set_load_force.restype = C.c_int
        lib.orc_set_load_force.argtypes = [vp, C.c_int32, d]
        _lib = lib
    return _lib


def _geoms_c(geoms):
    if not geoms:
        return None, 0, None
    arr = (_Geom * len(geoms))(*[g.to_c() for g in geoms])
    return C.cast(arr, C.c_void_p), len(geoms), arr


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def detect(x, r, ids, geoms=(), cap=None):
    """Brute-force contact set: arrays (key_a, key_b, delta), sorted by key."""
    lib = load()
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    r = np.ascontiguousarray(r, dtype=np.float64)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    n = r.shape[0]
    gp, ng, keep = _geoms_c(list(geoms))
    cap = cap or max(16, 16 * n)
    while True:
        a = np.zeros(cap, np.int32); b = np.zeros(cap, np.int32); dl = np.zeros(cap, np.float64)
        m = lib.orc_detect(n, x, r, ids, ng, gp, cap, a, b, dl)
        if m <= cap:
            return a[:m], b[:m], dl[:m]
        cap = int(m)


class Oracle:
    """A stepping FP64 simulation.  State arrays are float64 numpy arrays."""

    def __init__(self, params: OracleParams, x, r, v=None, w=None, ids=None, geoms=(),
                 inv_m=None, inv_I=None):
        self.lib = load()
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        n = x.shape[0]
        self.n = n
        r = np.ascontiguousarray(r, dtype=np.float64)
        v = np.zeros((n, 3)) if v is None else np.ascontiguousarray(v, dtype=np.float64)
        w = np.zeros((n, 3)) if w is None else np.ascontiguousarray(w, dtype=np.float64)
        ids = np.arange(n, dtype=np.int32) if ids is None else np.ascontiguousarray(ids, np.int32)
        self.geoms = list(geoms)
        gp, ng, keep = _geoms_c(self.geoms)
        self._params = params.to_c()
        im = None if inv_m is None else np.ascontiguousarray(inv_m, dtype=np.float64)
        iI = None if inv_I is None else np.ascontiguousarray(inv_I, dtype=np.float64)
        self.h = self.lib.orc_create(C.byref(self._params), n, x.reshape(-1), r, v.reshape(-1),
                                     w.reshape(-1), ids, _ptr(im), _ptr(iI), ng, gp)
        self.ng = ng

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def step(self, nsteps=1):
        if self.lib.orc_step(self.h, int(nsteps)) != 0:
            raise ValueError("the PGS solver does not take load-driven groups")

    def colours(self):
        """Colours of the last PGS step (0 for Jacobi)."""
        return int(self.lib.orc_colours(self.h))

    def impacts(self):
        """Impacting contacts of the last step (0: no impact stage ran)."""
        return int(self.lib.orc_impacts(self.h))

    def state(self):
        x = np.zeros((self.n, 3)); v = np.zeros((self.n, 3)); w = np.zeros((self.n, 3))
        self.lib.orc_get_state(self.h, _ptr(x), _ptr(v), _ptr(w))
        return x, v, w

    def set_state(self, x=None, v=None, w=None):
        c = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        xx, vv, ww = c(x), c(v), c(w)
        self.lib.orc_set_state(self.h, _ptr(xx), _ptr(vv), _ptr(ww))

    def set_geom_velocity(self, g, v, w=(0.0, 0.0, 0.0)):
        self.lib.orc_set_geom_velocity(self.h, int(g), np.asarray(v, np.float64),
                                       np.asarray(w, np.float64))

    def geom(self, g) -> Geom:
        out = _Geom()
        self.lib.orc_get_geom(self.h, int(g), C.byref(out))
        return Geom.from_c(out)

    def geom_force(self, g):
        f = np.zeros(3); t = np.zeros(3)
        self.lib.orc_get_geom_force(self.h, int(g), f, t)
        return f, t

    def contacts(self):
        """(key_a, key_b, lam7, delta, normal) of the last step, sorted by key."""
        m = self.lib.orc_get_contacts(self.h, 0, None, None, None, None, None)
        a = np.zeros(m, np.int32); b = np.zeros(m, np.int32)
        lam = np.zeros((m, 7)); dl = np.zeros(m); nn = np.zeros((m, 3))
        self.lib.orc_get_contacts(self.h, m, _ptr(a), _ptr(b), _ptr(lam), _ptr(dl), _ptr(nn))
        return a, b, lam, dl, nn

    def set_load(self, geoms, mass, force, dof=4):
        """Bind primitives into one load-driven rigid group (orc_set_load)."""
        g = np.ascontiguousarray(geoms, np.int32)
        if self.lib.orc_set_load(self.h, len(g), g, float(mass), np.asarray(force, np.float64), int(dof)) != 0:
            raise ValueError("orc_set_load rejected its arguments")

    def set_load_force(self, g, force):
        """New external force of the group holding primitive g (orc_set_load_force)."""
        if self.lib.orc_set_load_force(self.h, int(g), np.asarray(force, np.float64)) != 0:
            raise ValueError("primitive %d is in no load-driven group" % g)

    def set_warmstart(self, key_a, key_b, lam7):
        ka = np.ascontiguousarray(key_a, np.int32); kb = np.ascontiguousarray(key_b, np.int32)
        lam = np.ascontiguousarray(lam7, np.float64).reshape(-1)
        self.lib.orc_set_warmstart(self.h, len(ka), ka, kb, lam)
