"""Pin of the oracle's projected Jacobi limit against the exact solution of a
tiny complementarity problem (Sec. 2.2, Eqs. 2 and 5), found by enumerating
active sets.

Without friction and rolling resistance the tangential and rolling impulses
are projected to zero and one step reduces to the normal rows:
    w = (G M^-1 G^T + Sigma) p + (G v* - b) >= 0,  p >= 0,  p . w = 0,
with G the unit normals (from b to a, particles' arms along n), M the masses
(the split masses of the iteration only precondition it), v* = v + dt g, and
each row's compliance Sigma and right side b of the SPOOK stepper for the Hertz
mapping (the physical-impulse form: g = -delta^e_H, J = e_H max(delta,
delta_floor)^(e_H - 1), Sigma = 4 Y eps / (dt^2 J^2), b = -(4/dt) Y g / J + Y G v,
Y = 1 / (1 + 4 d)).  With three contacts the 2^3 active sets are tried; exactly
one is complementary (the matrix is positive definite), and the oracle's
iterate after many sweeps must equal it.  A contact that separates (p = 0)
and two that push make the active set non-trivial.
"""
import itertools
import math

import numpy as np

from oracle import Geom, Oracle, OracleParams
from oracle.binding import PLANE

RHO, E, NU, DT, EH, D, FLOOR = 2600.0, 1e9, 0.15, 1e-5, 1.25, 4.5, 1e-8


def kn(d_eff):
    estar = 1.0 / (2 * (1 - NU ** 2) / E)
    return estar * math.sqrt(d_eff) / 3.0


def row_constants(delta, k):
    ups = 1.0 / (1.0 + 4.0 * D)
    eps = EH / k
    J = EH * max(delta, FLOOR) ** (EH - 1.0)
    gap = -delta ** EH
    sigma = 4.0 * eps * ups / (DT * DT) / (J * J)
    b_gap = (-(4.0 / DT) * ups * gap) / J
    return sigma, b_gap, ups


def test_jacobi_limit_equals_enumerated_lcp_solution():
    r = 5e-3
    dA_floor, dA_wall, dAB = 2e-6, 1.5e-6, 1e-6
    xA = np.array([r - dA_wall, 0.0, r - dA_floor])          # touching the wall x = 0 and the floor z = 0
    dx = 2e-5                                                 # clear of the wall
    xB = xA + np.array([dx, 0.0, math.sqrt((2 * r - dAB) ** 2 - dx * dx)])   # on top of A
    vA = np.array([-0.02, 0.0, -0.01])                        # into the wall and the floor
    vB = np.array([0.0, 0.0, 0.05])                           # leaving A
    p = OracleParams(rho=RHO, E=E, nu=NU, mu_t=0.0, mu_r=0.0, e_H=EH, damp_steps=D, dt=DT, n_it=20000,
                     gravity=(0.0, 0.0, -9.81), delta_floor=FLOOR)
    floor = Geom(PLANE, c=(0, 0, 0), E=E, nu=NU, mu_t=0.0, mu_r=0.0)
    wall = Geom(PLANE, c=(0, 0, 0), R=(0, 0, 1, 0, 1, 0, -1, 0, 0), E=E, nu=NU, mu_t=0.0, mu_r=0.0)  # normal +x
    o = Oracle(p, np.stack([xA, xB]), np.array([r, r]), v=np.stack([vA, vB]), geoms=[floor, wall])
    o.step(1)
    ka, kb, lam, dl, nn = o.contacts()
    assert len(ka) == 3

    m = RHO * 4 / 3 * math.pi * r ** 3
    g = np.array([0.0, 0.0, -9.81])
    vs = np.concatenate([vA + DT * g, vB + DT * g])            # v* of A, B
    v0 = np.concatenate([vA, vB])
    # rows in the oracle's key order: (A, B), (A, floor = -1), (A, wall = -2)
    rows, sig, b = [], [], []
    for a_id, b_id, delta in zip(ka, kb, dl):
        Gr = np.zeros(6)
        if b_id >= 0:
            n = (xA - xB) / np.linalg.norm(xA - xB)               # from B to A
            Gr[:3], Gr[3:] = n, -n
            k = kn(2 * r * 2 * r / (4 * r))
        else:
            n = np.array([0.0, 0.0, 1.0]) if b_id == -1 else np.array([1.0, 0.0, 0.0])
            Gr[:3] = n
            k = kn(2 * r)
        s_, bg, ups = row_constants(delta, k)
        rows.append(Gr)
        sig.append(s_)
        b.append(bg + ups * Gr @ v0)
    G = np.array(rows)
    A = G @ G.T / m + np.diag(sig)
    q = G @ vs - np.array(b)
    # enumerate the active sets
    sols = []
    for act in itertools.product([False, True], repeat=3):
        S = np.array(act)
        pS = np.zeros(3)
        if S.any():
            pS[S] = np.linalg.solve(A[np.ix_(S, S)], -q[S])
        w = A @ pS + q
        if (pS >= -1e-15).all() and (w[~S] >= -1e-12).all():
            sols.append(pS)
    assert len(sols) == 1
    exact = sols[0]
    assert (exact > 0).sum() == 2 and (exact == 0).sum() == 1     # one contact separates
    assert np.abs(lam[:, 0] - exact).max() < 1e-9 * np.abs(exact).max()
    assert np.abs(lam[:, 1:]).max() == 0.0                          # no friction, no rolling
