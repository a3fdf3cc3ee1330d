"""Pins of the oracle's contact detection.

Sphere-sphere: the O(N^2) brute force is the definition; it is checked against
an independent KD-tree candidate search (scipy) with the same predicate.
Sphere-geometry: the closed-form closest points are checked against dense
sampling of the primitive's surface.
"""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from oracle import Geom
from oracle.binding import PLANE, BOX, CYLINDER


@pytest.mark.parametrize("seed,n", [(1, 300), (2, 1000)])
def test_pairs_match_kdtree(seed, n):
    rng = np.random.default_rng(seed)
    r = rng.uniform(2e-3, 16e-3, n)       # size ratio 8, as in refined beds
    x = rng.uniform(0, 0.15, (n, 3))
    ids = rng.permutation(n).astype(np.int32)
    a, b, dl = oracle.detect(x, r, ids)
    tree = cKDTree(x)
    cand = tree.query_pairs(2 * r.max(), output_type="ndarray")
    d = np.linalg.norm(x[cand[:, 0]] - x[cand[:, 1]], axis=1)
    hit = cand[d < r[cand[:, 0]] + r[cand[:, 1]]]
    ref = {(min(ids[i], ids[j]), max(ids[i], ids[j])) for i, j in hit}
    got = set(zip(a.tolist(), b.tolist()))
    assert got == ref
    assert len(got) == len(a)                      # no duplicates
    assert (a < b).all()
    # overlaps: r_a + r_b - |x_a - x_b|
    inv = np.argsort(ids)
    ia, ib = inv[a], inv[b]
    ref_dl = r[ia] + r[ib] - np.linalg.norm(x[ia] - x[ib], axis=1)
    assert np.allclose(dl, ref_dl, rtol=0, atol=1e-15)
    assert (dl > 0).all()


def rot(ax, ang):
    ax = np.asarray(ax, float) / np.linalg.norm(ax)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def sample_surface(kind, he, m=120):
    """Dense sample of the primitive's surface in local coordinates."""
    pts = []
    if kind == BOX:
        u = np.linspace(-1, 1, m)
        U, V = np.meshgrid(u, u)
        U, V = U.ravel(), V.ravel()
        for k in range(3):
            i, j = [q for q in range(3) if q != k]
            for s in (-1, 1):
                p = np.zeros((U.size, 3))
                p[:, k] = s * he[k]
                p[:, i] = U * he[i]
                p[:, j] = V * he[j]
                pts.append(p)
    else:
        R, H = he[0], he[2]
        th = np.linspace(0, 2 * np.pi, 4 * m, endpoint=False)
        z = np.linspace(-H, H, m)
        T, Z = np.meshgrid(th, z)
        pts.append(np.stack([R * np.cos(T.ravel()), R * np.sin(T.ravel()), Z.ravel()], 1))
        rr = np.linspace(0, R, m)
        RR, TT = np.meshgrid(rr, th)
        for s in (-1, 1):
            pts.append(np.stack([RR.ravel() * np.cos(TT.ravel()), RR.ravel() * np.sin(TT.ravel()),
                                 np.full(RR.size, s * H)], 1))
    return np.concatenate(pts)


def inside(kind, he, q):
    if kind == BOX:
        return (np.abs(q) <= he).all()
    return q[0] ** 2 + q[1] ** 2 <= he[0] ** 2 and abs(q[2]) <= he[2]


@pytest.mark.parametrize("kind,he", [(BOX, (0.03, 0.02, 0.01)), (CYLINDER, (0.05, 0.0, 0.005))])
def test_geometry_overlap_matches_surface_sampling(kind, he):
    rng = np.random.default_rng(11)
    Rm = rot((1, 2, 3), 0.7)
    c = np.array([0.1, -0.05, 0.2])
    g = Geom(kind, c=tuple(c), R=tuple(Rm.reshape(-1)), he=he)
    surf = sample_surface(kind, np.array(he))
    h = 2.0 / 120 * max(he) * 1.5            # sampling resolution bound
    n = 400
    q = rng.uniform(-1.6, 1.6, (n, 3)) * np.array([max(he[0], 0.01), max(he[1], he[0], 0.01), max(he[2], 0.01)])
    xw = c + q @ Rm.T
    r = rng.uniform(3e-3, 12e-3, n)
    a, b, dl = oracle.detect(xw, r, np.arange(n, dtype=np.int32), [g])
    geo = b == -1                          # keep sphere-geometry contacts only
    got = dict(zip(a[geo].tolist(), dl[geo].tolist()))
    checked = 0
    for i in range(n):
        dist = np.linalg.norm(surf - q[i], axis=1).min()
        ref = r[i] + dist if inside(kind, np.array(he), q[i]) else r[i] - dist
        if abs(ref) < 2 * h:
            continue                       # too close to the sampling resolution
        if ref > 0:
            assert i in got, (i, ref)
            assert abs(got[i] - ref) < 2 * h
            checked += 1
        else:
            assert i not in got
    assert checked > 20


def test_plane_overlap():
    Rm = rot((1, 0, 0), 0.3)
    g = Geom(PLANE, c=(0.0, 0.0, 0.1), R=tuple(Rm.reshape(-1)))
    nrm = Rm[:, 2]
    x = np.array([[0.0, 0.0, 0.1], [0.05, 0.02, 0.1]]) + np.array([[0.004], [0.02]]) * nrm
    r = np.array([0.005, 0.01])
    a, b, dl = oracle.detect(x, r, np.arange(2, dtype=np.int32), [g])
    assert a.tolist() == [0] and b.tolist() == [-1]
    assert dl[0] == pytest.approx(0.001, abs=1e-15)
