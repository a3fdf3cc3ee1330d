"""Pins of the oracle's spinning kinematic primitives (Sec. 2.2: the motor
constraint drives geometry with a prescribed linear and angular velocity).

A primitive moving with velocity v and angular velocity w about its centre c
moves its surface point q at v + w x (q - c).  The contact rows take that
velocity at the contact point (the middle of the overlap), and the rolling and
twisting rows take the relative angular velocity w_sphere - w.  Each test below
fixes one part of this against mechanics or a library routine:

- a turntable (a floor spinning about its normal) under a sphere that cannot
  rotate drags it at mu_t g in the direction the floor moves under it, until
  the sphere rides with the floor, v = w x (x - c) (belt problem);
- a sphere on the turntable's axis is spun up by the twisting row at
  mu_r r m g / I until it turns with the table;
- one step against a flipper (a wall spinning about an axis in its own plane)
  equals one step against the same wall translating with the velocity its
  surface has at the contact point (lever from the centre to the middle of
  the overlap, sign of w x lever), with rolling resistance off;
- the pose update over many steps equals scipy's rotation by the accumulated
  rotation vector (Rodrigues' formula, for a constant w).
"""
import math

import numpy as np
import pytest

from oracle import Geom, Oracle, OracleParams
from oracle.binding import BOX, PLANE

E, NU, RHO, G = 1e9, 0.15, 2600.0, 9.81
R0 = 5e-3
DT = 1e-5


def mass(r=R0):
    return RHO * 4 / 3 * math.pi * r ** 3


def kn_wall(r=R0):
    estar = 1.0 / ((1 - NU ** 2) / E + (1 - NU ** 2) / E)
    return estar * math.sqrt(2 * r) / 3.0


def turntable(omega, rho, mu_t, mu_r, rotate, n_it=60):
    m = mass()
    d0 = (m * G / kn_wall()) ** (2 / 3)      # static overlap: start at rest on the table
    p = OracleParams(rho=RHO, E=E, nu=NU, mu_t=mu_t, mu_r=mu_r, dt=DT, n_it=n_it,
                     gravity=(0, 0, -G), delta_floor=1e-10)
    table = Geom(PLANE, c=(0, 0, 0), w=(0.0, 0.0, omega), E=E, nu=NU, mu_t=mu_t, mu_r=mu_r)
    inv_I = None if rotate else np.zeros(1)
    return Oracle(p, np.array([[rho, 0.0, R0 - d0]]), np.array([R0]), geoms=[table], inv_I=inv_I)


def test_turntable_drags_sphere_at_mu_g_then_carries_it():
    omega, rho, mu = 2.0, 0.05, 0.3
    o = turntable(omega, rho, mu, 0.0, rotate=False)
    o.step(200)
    _, v0, _ = o.state()
    o.step(500)
    _, v1, _ = o.state()
    a = (v1[0] - v0[0]) / (500 * DT)
    # the table moves at w x (x - c) = (0, omega rho, 0) under the sphere
    assert abs(np.linalg.norm(a[:2]) / (mu * G) - 1) < 2e-3
    assert a[1] > 0 and abs(a[0]) < 2e-2 * abs(a[1])
    # slip ends after omega rho / (mu g); then the sphere rides with the table
    t_stick = omega * rho / (mu * G)
    o.step(int(1.5 * t_stick / DT))
    x, v, _ = o.state()
    carried = np.cross([0.0, 0.0, omega], x[0])
    assert np.linalg.norm(v[0, :2] - carried[:2]) < 1e-3 * np.linalg.norm(carried)
    # and turns with it: polar angle advances at omega
    phi0 = math.atan2(x[0, 1], x[0, 0])
    o.step(2000)
    x2, _, _ = o.state()
    phi1 = math.atan2(x2[0, 1], x2[0, 0])
    assert abs((phi1 - phi0) / (2000 * DT) / omega - 1) < 1e-3
    # the table's pose: a plane spun about its normal keeps its normal
    g = o.geom(0)
    assert np.allclose(np.array(g.R).reshape(3, 3)[:, 2], [0, 0, 1], atol=1e-15)


def test_turntable_twists_sphere_on_its_axis():
    """On the axis the table's surface does not translate: only the twisting
    row acts, with torque bounded by mu_r r_eff p_n (Eq. 7, r_eff = r for a
    primitive), so the spin grows at mu_r r m g / I until it equals omega."""
    omega, mu_r = 2.0, 0.1
    o = turntable(omega, 0.0, 0.5, mu_r, rotate=True, n_it=120)
    o.step(20)
    _, _, w0 = o.state()
    o.step(100)
    _, _, w1 = o.state()
    m = mass()
    I = 0.4 * m * R0 ** 2
    alpha = (w1[0, 2] - w0[0, 2]) / (100 * DT)
    assert abs(alpha / (mu_r * R0 * m * G / I) - 1) < 2e-3
    o.step(int(1.5 * omega * I / (mu_r * R0 * m * G) / DT))
    x, v, w = o.state()
    assert abs(w[0, 2] / omega - 1) < 1e-4
    assert np.abs(v[0]).max() < 1e-6 and np.abs(w[0, :2]).max() < 1e-6


def flipper_step(spin):
    """One step of a sphere pressed into a wall (normal +x, through c) that
    spins at w (spin=True) or translates with the velocity its surface has at
    the middle of the overlap (spin=False)."""
    c = np.array([0.0, 0.05, -0.1])             # on the wall plane x = 0
    w = np.array([0.3, 0.5, -0.2])
    delta = 2e-5
    xs = np.array([R0 - delta, 0.012, 0.03])      # sphere centre, wall plane x = 0
    n = np.array([1.0, 0.0, 0.0])
    q_mid = xs - (R0 - delta / 2) * n             # middle of the overlap
    v_point = np.cross(w, q_mid - c)
    p = OracleParams(rho=RHO, E=E, nu=NU, mu_t=0.4, mu_r=0.0, dt=DT, n_it=80,
                     gravity=(0, 0, -G), delta_floor=1e-10)
    Rm = (0, 0, 1, 0, 1, 0, -1, 0, 0)               # local z (the normal) = world x
    if spin:
        wall = Geom(PLANE, c=tuple(c), R=Rm, v=(0, 0, 0), w=tuple(w), E=E, nu=NU, mu_t=0.4, mu_r=0.0)
    else:
        wall = Geom(PLANE, c=tuple(c), R=Rm, v=tuple(v_point), w=(0, 0, 0), E=E, nu=NU, mu_t=0.4, mu_r=0.0)
    o = Oracle(p, xs[None, :], np.array([R0]), v=np.array([[0.0, 0.02, 0.0]]), w=np.array([[0.0, 0.0, 3.0]]),
               geoms=[wall])
    o.step(1)
    x, v, ww = o.state()
    lam = o.contacts()[2]
    f, t = o.geom_force(0)
    return v[0], ww[0], lam[0], f, v_point


def test_spinning_wall_acts_through_its_contact_point_velocity():
    v_s, w_s, lam_s, f_s, vp = flipper_step(True)
    v_t, w_t, lam_t, f_t, _ = flipper_step(False)
    # the spin pushes (normal part of the point velocity) and drags (tangential part)
    assert vp[0] > 0 and np.linalg.norm(vp[1:]) > 0.01
    assert lam_s[0] > 0 and np.linalg.norm(lam_s[1:4]) > 0
    scale = np.abs(lam_t).max()
    assert np.abs(lam_s - lam_t).max() < 1e-12 * scale
    assert np.abs(v_s - v_t).max() < 1e-12 * np.abs(v_t).max()
    assert np.abs(w_s - w_t).max() < 1e-12 * np.abs(w_t).max()
    assert np.abs(f_s - f_t).max() < 1e-12 * np.abs(f_t).max()


def test_pose_update_matches_rotation_vector():
    Rotation = pytest.importorskip("scipy.spatial.transform").Rotation
    w = np.array([0.3, -0.5, 0.8])
    v = np.array([0.01, 0.02, -0.03])
    R0m = Rotation.from_euler("xyz", [0.2, -0.4, 1.1]).as_matrix()
    c0 = np.array([0.4, -0.2, 0.3])
    box = Geom(BOX, c=tuple(c0), R=tuple(R0m.reshape(-1)), he=(0.02, 0.03, 0.01), v=tuple(v), w=tuple(w),
               E=E, nu=NU, mu_t=0.3, mu_r=0.0)
    p = OracleParams(rho=RHO, E=E, nu=NU, mu_t=0.3, mu_r=0.0, dt=DT, n_it=4, gravity=(0, 0, 0))
    o = Oracle(p, np.array([[5.0, 5.0, 5.0]]), np.array([R0]), geoms=[box])   # a sphere far away
    steps = 3000
    o.step(steps)
    g = o.geom(0)
    R = np.array(g.R).reshape(3, 3)
    R_ref = Rotation.from_rotvec(steps * DT * w).as_matrix() @ R0m
    assert np.abs(R - R_ref).max() < 1e-12
    assert np.abs(R.T @ R - np.eye(3)).max() < 1e-12
    # 3000 rounded additions of dt v
    assert np.allclose(g.c, c0 + steps * DT * v, rtol=0, atol=1e-12)
