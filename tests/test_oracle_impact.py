"""Pins of the oracle's Newton impact stage (Sec. 2.2: high-velocity impacts
follow Newton's impact law while the other kinematic constraints are kept).

Reading: a contact approaching faster than the threshold is an impact; when a
step has one, normal impulses of every contact are solved on the velocity
level with u+ >= -e u- for impacts and u+ >= 0 for the other contacts, from
the velocities at the start of the step, before the SPOOK solve.

The overlaps here are 1e-9 m, so the SPOOK rows that follow add no impulse
(their gap term asks for ~1e-8 m/s, bounded in the test, and contacts that
separate get none): the step's
velocities are the impact stage's, and they have closed forms -- Newton's
restitution law for one contact, the simultaneous-impact solution for a chain.
"""
import math

import numpy as np
import pytest

from oracle import Geom, Oracle, OracleParams
from oracle.binding import PLANE

R = 5e-3
RHO = 2600.0
DELTA = 1e-9


def mass(r):
    return RHO * 4.0 / 3.0 * math.pi * r ** 3


def gap_speed(h=1e-5, d=4.5, e_H=1.25, floor=1e-8):
    """Separation speed the SPOOK row of a resting 1e-9 m overlap asks for:
    (4/dt) Ups delta^e_H / J, J = e_H max(delta, floor)^(e_H - 1)."""
    ups = 1.0 / (1.0 + 4.0 * d)
    return (4.0 / h) * ups * DELTA ** e_H / (e_H * max(DELTA, floor) ** (e_H - 1.0))


def params(e, v_imp=0.1, n_it=2000, g=0.0):
    return OracleParams(mu_t=0.0, mu_r=0.0, n_it=n_it, gravity=(0.0, 0.0, -g) if g else (0.0, 0.0, 0.0),
                        restitution=e, impact_speed=v_imp)


def pair(ra, rb, va, vb, e, v_imp=0.1):
    x = np.array([[0.0, 0.0, 0.0], [ra + rb - DELTA, 0.0, 0.0]])
    v = np.array([[va, 0.0, 0.0], [vb, 0.0, 0.0]])
    o = Oracle(params(e, v_imp), x, np.array([ra, rb]), v=v)
    o.step(1)
    return o


@pytest.mark.parametrize("e", [0.0, 0.5, 1.0])
def test_head_on_equal_masses_newton_law(e):
    V = 1.0
    o = pair(R, R, V / 2, -V / 2, e)
    assert o.impacts() == 1
    v = o.state()[1][:, 0]
    # relative normal velocity reversed and scaled by e, momentum kept; at
    # e = 0 the pair rests and its SPOOK row pushes the overlap apart
    tol = 1e-12 + (1.01 * gap_speed() if e == 0.0 else 0.0)
    assert abs((v[1] - v[0]) - e * V) < tol
    assert abs(v[0] + v[1]) < 1e-12 * V
    assert abs(v[0] - (-e * V / 2)) < tol


def test_head_on_unequal_masses():
    ra, rb, va, vb, e = 5e-3, 7e-3, 1.5, -0.25, 0.7
    o = pair(ra, rb, va, vb, e)
    ma, mb = mass(ra), mass(rb)
    # Newton: v_a' = (ma va + mb vb - mb e (va - vb)) / (ma + mb), and symmetrically
    ea = (ma * va + mb * vb - mb * e * (va - vb)) / (ma + mb)
    eb = (ma * va + mb * vb + ma * e * (va - vb)) / (ma + mb)
    v = o.state()[1][:, 0]
    assert abs(v[0] - ea) < 1e-9 and abs(v[1] - eb) < 1e-9


def test_below_threshold_is_untouched_bit_for_bit():
    x = np.array([[0.0, 0.0, 0.0], [2 * R - 1e-6, 0.0, 0.0]])
    v = np.array([[0.04, 0.0, 0.0], [-0.04, 0.0, 0.0]])
    out = []
    for v_imp in (0.0, 0.1):
        o = Oracle(params(0.5, v_imp, n_it=50), x, np.array([R, R]), v=v)
        o.step(3)
        assert o.impacts() == 0
        out.append(o.state())
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_sphere_on_floor_rebound_and_floor_impulse():
    V, e, g, h = 2.0, 0.8, 9.81, 1e-5
    floor = Geom(PLANE, c=(0, 0, 0), mu_t=0.0, mu_r=0.0)
    x = np.array([[0.0, 0.0, R - DELTA]])
    o = Oracle(params(e, g=g), x, np.array([R]), v=np.array([[0.0, 0.0, -V]]), geoms=[floor])
    o.step(1)
    assert o.impacts() == 1
    vz = o.state()[1][0, 2]
    # rebound e V, then the free flight of the step (the SPOOK row stays inactive)
    assert abs(vz - (e * V - g * h)) < 1e-9
    # the floor takes the impact impulse -(1 + e) m V (as force: / dt) in the same step
    f, _ = o.geom_force(0)
    assert abs(f[2] / (-(1 + e) * mass(R) * V / h) - 1) < 1e-9


@pytest.mark.parametrize("e,expect", [(0.0, (1 / 3, 1 / 3, 1 / 3)), (1.0, (-1 / 3, 2 / 3, 2 / 3))])
def test_chain_keeps_the_other_constraints(e, expect):
    # A hits B, which touches C at rest: the B-C contact is not an impact but
    # keeps u+ >= 0.  e = 0: all three move on together at V/3.  e = 1: A-B
    # separate at V and B, C move together: A -V/3, B and C 2V/3.
    V = 1.0
    x = np.array([[0.0, 0.0, 0.0], [2 * R - DELTA, 0.0, 0.0], [4 * R - 2 * DELTA, 0.0, 0.0]])
    v = np.array([[V, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    o = Oracle(params(e), x, np.full(3, R), v=v)
    o.step(1)
    assert o.impacts() == 1
    got = o.state()[1][:, 0]
    assert np.abs(got - np.array(expect) * V).max() < 1e-6 * V
