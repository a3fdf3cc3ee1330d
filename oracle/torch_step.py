"""FP64 PyTorch restatement of the oracle step, differentiable by autograd.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/).  It gives the reference
gradient of a weighted sum of geometry forces with respect to the contact
stiffness scale, the friction coefficient and the rolling-resistance
coefficient, on the contact sets of the forward run ("fixed topology per
step"): the contact set of every step comes from the C oracle's brute-force
detection and is not differentiated; everything else is.

The step is the same algorithm as oracle.c (Sec. 2.2 of the paper, SPOOK rows,
N_it projected Jacobi sweeps with mass splitting, x += dt v), written with
world-frame tangential vectors instead of a 2D tangent basis (the two agree:
the tangential impulse always lies in the tangent plane).  Geometry: planes,
oriented boxes and cylinders that translate kinematically (no spin); the
closest point takes the same cases as oracle.c (face, edge, corner, side,
rim, centre inside), decided on the forward values and differentiated within
the case.  Its forward values are pinned against oracle.c by the tests.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as _b


def _cross(a, b):
    return torch.cross(a, b, dim=-1)


def _dot(a, b):
    return (a * b).sum(-1)


def _norm(a):
    """|a| with a zero (not NaN) derivative at a = 0."""
    q = _dot(a, a)
    pos = q > 0
    return torch.where(pos, torch.sqrt(torch.where(pos, q, torch.ones_like(q))), torch.zeros_like(q))


def _geom_contact(g, x, c, r):
    """Unit normal (from the primitive to the sphere centre) and overlap of a
    sphere of radius r at x with primitive g whose centre or reference point
    is c; the case decisions of oracle.c's closest point, taken on the values,
    the results differentiable in x and c."""
    R = torch.tensor(g.R, dtype=torch.float64).reshape(3, 3)   # column k = local axis k
    if g.type == _b.PLANE:
        nz = R[:, 2]
        return nz, r - _dot(nz, x - c)
    q = R.T @ (x - c)
    qd = q.detach().numpy()
    if g.type == _b.BOX:
        he = torch.tensor(g.he, dtype=torch.float64)
        cl = torch.maximum(torch.minimum(q, he), -he)
        e = q - cl
        ee = float(_dot(e, e).detach())
        if ee > 0.0:
            d = torch.sqrt(_dot(e, e))
            return R @ (e / d), r - d
        depth = np.asarray(g.he) - np.abs(qd)
        kb = int(np.argmin(depth))            # first minimum, as the C loop keeps
        sg = -1.0 if qd[kb] < 0.0 else 1.0
        nl = torch.zeros(3, dtype=torch.float64)
        nl[kb] = sg
        return R @ nl, r + (g.he[kb] - sg * q[kb])
    Rc, H = g.he[0], g.he[2]
    rho2 = q[0] * q[0] + q[1] * q[1]
    if float(rho2.detach()) > Rc * Rc:
        rho = torch.sqrt(rho2)
        clxy = q[:2] * (Rc / rho)
    else:
        clxy = q[:2]
    clz = torch.clamp(q[2], -H, H)
    e = torch.cat([q[:2] - clxy, (q[2] - clz).reshape(1)])
    ee = float(_dot(e, e).detach())
    if ee > 0.0:
        d = torch.sqrt(_dot(e, e))
        return R @ (e / d), r - d
    rho = torch.sqrt(rho2)
    da = H - abs(qd[2])
    dr = Rc - float(rho.detach())
    if da <= dr:
        sg = -1.0 if qd[2] < 0.0 else 1.0
        return R @ torch.tensor([0.0, 0.0, sg], dtype=torch.float64), r + (H - sg * q[2])
    if float(rho.detach()) > 0.0:
        nl = torch.cat([q[:2] / rho, torch.zeros(1, dtype=torch.float64)])
    else:
        nl = torch.tensor([1.0, 0.0, 0.0], dtype=torch.float64)
    return R @ nl, r + (Rc - rho)


class TorchStepper:
    """params: OracleParams (dt, n_it, e_H, damp_steps, E, nu, rho, eps_reg,
    delta_floor, gravity); theta = (kn_scale, mu_t, mu_r) as torch tensors;
    planes: list of oracle Geom (plane, box or cylinder; kinematic translation
    allowed, no spin).  Particle-primitive contacts use the primitive's own
    mu_t, mu_r (not differentiated)."""

    def __init__(self, params, r, ids, planes, inv_m=None, inv_I=None):
        self.p = params
        self.r = torch.as_tensor(np.asarray(r, np.float64))
        self.ids = np.asarray(ids, np.int32)
        self.planes = list(planes)
        m = params.rho * 4.0 / 3.0 * np.pi * self.r ** 3
        self.inv_m = torch.as_tensor(inv_m, dtype=torch.float64) if inv_m is not None else 1.0 / m
        self.inv_I = torch.as_tensor(inv_I, dtype=torch.float64) if inv_I is not None else 1.0 / (0.4 * m * self.r ** 2)

    def _contacts(self, x, plane_pos):
        """Contact keys of the oracle's detection at positions x, with every
        plane where it stands at the start of the step (no gradient)."""
        geoms = [_b.Geom(g.type, tuple(float(q) for q in pp), g.R, g.he, g.v, g.w, g.E, g.nu, g.mu_t, g.mu_r)
                 for g, pp in zip(self.planes, plane_pos)]
        ka, kb, _ = _b.detect(x.detach().numpy(), self.r.numpy(), self.ids, geoms)
        inv = np.empty(self.ids.max() + 1 if len(self.ids) else 1, np.int64)
        inv[self.ids] = np.arange(len(self.ids))
        ss = kb >= 0
        a = inv[ka[ss]]
        b = inv[kb[ss]]
        ga = inv[ka[~ss]]
        gg = -kb[~ss] - 1
        return (ka, kb), a, b, ga, gg

    def step(self, x, v, w, theta, warm, plane_pos):
        """One step.  x, v, w: (N,3) tensors; warm: dict key -> (7,) tensor of
        world-frame impulses; plane_pos: list of plane reference points (tensors,
        moved kinematically).  Returns x', v', w', warm', forces (G,3), keys."""
        P = self.p
        h, ups = P.dt, 1.0 / (1.0 + 4.0 * P.damp_steps)
        kns, mu_t, mu_r = theta
        keys, a, b, ga, gg = self._contacts(x, plane_pos)
        nb = len(a)
        ng_c = len(ga)
        N = x.shape[0]
        cnt = torch.zeros(N, dtype=torch.float64)
        cnt.index_add_(0, torch.as_tensor(a), torch.ones(nb, dtype=torch.float64))
        cnt.index_add_(0, torch.as_tensor(b), torch.ones(nb, dtype=torch.float64))
        cnt.index_add_(0, torch.as_tensor(ga), torch.ones(ng_c, dtype=torch.float64))
        A = torch.as_tensor(np.concatenate([a, ga]))          # body a of every contact
        Bsph = torch.as_tensor(b)
        nc = nb + ng_c
        # ---- geometry of the rows ----
        d = x[a] - x[b]
        dist = torch.sqrt(_dot(d, d))
        n_s = d / dist[:, None]
        ra, rb = self.r[a], self.r[b]
        delta_s = ra + rb - dist
        Estar_ss = 1.0 / (2 * (1 - P.nu ** 2) / P.E)
        dstar_s = 1.0 / (1.0 / (2 * ra) + 1.0 / (2 * rb))
        reff_s = 2 * ra * rb / (ra + rb)
        n_g, delta_g, Estar_g, mut_g, mur_g, vg = [], [], [], [], [], []
        for k in range(ng_c):
            pl = self.planes[gg[k]]
            nk, dk = _geom_contact(pl, x[ga[k]], plane_pos[gg[k]], self.r[ga[k]])
            n_g.append(nk)
            delta_g.append(dk)
            Estar_g.append(1.0 / ((1 - P.nu ** 2) / P.E + (1 - pl.nu ** 2) / pl.E))
            mut_g.append(pl.mu_t)
            mur_g.append(pl.mu_r * float(self.r[ga[k]]))
            vg.append(torch.tensor(pl.v, dtype=torch.float64))
        if ng_c:
            n_g = torch.stack(n_g)
            delta_g = torch.stack(delta_g)
            vg = torch.stack(vg)
        else:
            n_g = torch.zeros((0, 3), dtype=torch.float64)
            delta_g = torch.zeros(0, dtype=torch.float64)
            vg = torch.zeros((0, 3), dtype=torch.float64)
        n = torch.cat([n_s, n_g])
        delta = torch.cat([delta_s, delta_g])
        la = self.r[A] - 0.5 * delta
        lb = torch.cat([rb - 0.5 * delta_s, torch.zeros(ng_c, dtype=torch.float64)])
        Estar = torch.cat([torch.full((nb,), Estar_ss, dtype=torch.float64),
                           torch.tensor(Estar_g, dtype=torch.float64)])
        dstar = torch.cat([dstar_s, 2 * self.r[ga] if ng_c else torch.zeros(0, dtype=torch.float64)])
        kn = kns * Estar * torch.sqrt(dstar) / 3.0
        eps = P.e_H / kn
        dfl = torch.clamp(delta, min=P.delta_floor)
        J = P.e_H * dfl ** (P.e_H - 1.0)
        gap = -delta ** P.e_H
        sig = 4.0 * eps * ups / (h * h) / (J * J)
        mt = torch.cat([mu_t.expand(nb), torch.tensor(mut_g, dtype=torch.float64)])
        mr = torch.cat([mu_r * reff_s, torch.tensor(mur_g, dtype=torch.float64)])
        # split masses
        ima, iIa = cnt[A] * self.inv_m[A], cnt[A] * self.inv_I[A]
        imb = torch.cat([cnt[Bsph] * self.inv_m[Bsph], torch.zeros(ng_c, dtype=torch.float64)])
        iIb = torch.cat([cnt[Bsph] * self.inv_I[Bsph], torch.zeros(ng_c, dtype=torch.float64)])
        sig_t = P.eps_reg * sig
        invDn = 1.0 / (ima + imb + sig)
        invDt = 1.0 / (ima + imb + la * la * iIa + lb * lb * iIb + sig_t)
        invDr = 1.0 / (iIa + iIb + sig_t)

        def rel_vel(vv, ww):
            va, wa = vv[A], ww[A]
            vb = torch.cat([vv[Bsph], vg])
            wb = torch.cat([ww[Bsph], torch.zeros((ng_c, 3), dtype=torch.float64)])
            return va - vb, wa, wb

        dv0, _, _ = rel_vel(v, w)
        rhs = (-(4.0 / h) * ups * gap) / J + ups * _dot(n, dv0)
        # ---- warm start ----
        ka, kb = keys
        kk = np.concatenate([np.stack([ka[kb >= 0], kb[kb >= 0]], 1), np.stack([ka[kb < 0], kb[kb < 0]], 1)])
        lam_n, lam_t, lam_r = [], [], []
        for c in range(nc):
            wv = warm.get((int(kk[c, 0]), int(kk[c, 1])))
            if wv is None:
                lam_n.append(torch.zeros((), dtype=torch.float64))
                lam_t.append(torch.zeros(3, dtype=torch.float64))
                lam_r.append(torch.zeros(3, dtype=torch.float64))
            else:
                pt = wv[1:4] - _dot(wv[1:4], n[c]) * n[c]
                lam_n.append(wv[0]); lam_t.append(pt); lam_r.append(wv[4:7])
        pn = torch.stack(lam_n) if nc else torch.zeros(0, dtype=torch.float64)
        pt = torch.stack(lam_t) if nc else torch.zeros((0, 3), dtype=torch.float64)
        pr = torch.stack(lam_r) if nc else torch.zeros((0, 3), dtype=torch.float64)
        vstar = v + torch.where(self.inv_m[:, None] > 0, h * torch.tensor(P.gravity, dtype=torch.float64), 0.0)

        def body(pn, pt, pr):
            Pimp = pn[:, None] * n + pt
            nxpt = _cross(n, pt)
            Ta = -la[:, None] * nxpt + pr
            Tb = -lb[:, None] * nxpt - pr
            accL = torch.zeros_like(v).index_add(0, A, Pimp)
            accA = torch.zeros_like(w).index_add(0, A, Ta)
            if nb:
                accL = accL.index_add(0, Bsph, -Pimp[:nb])
                accA = accA.index_add(0, Bsph, Tb[:nb])
            return vstar + self.inv_m[:, None] * accL, w + self.inv_I[:, None] * accA

        vv, ww = body(pn, pt, pr)
        for _ in range(P.n_it):
            dv, wa, wb = rel_vel(vv, ww)
            wn = _dot(n, dv) + sig * pn - rhs
            pn1 = torch.clamp(pn - invDn * wn, min=0.0)
            s = la[:, None] * wa + lb[:, None] * wb
            uc = dv - _cross(s, n)
            ut = uc - _dot(n, uc)[:, None] * n
            q = pt - invDt[:, None] * (ut + sig_t[:, None] * pt)
            qn = _norm(q)
            bt = mt * pn1
            sc = torch.where(qn > bt, bt / torch.where(qn > 0, qn, torch.ones_like(qn)), torch.ones_like(qn))
            pt1 = q * sc[:, None]
            qr = pr - invDr[:, None] * ((wa - wb) + sig_t[:, None] * pr)
            qrn = _norm(qr)
            br = mr * pn1
            scr = torch.where(qrn > br, br / torch.where(qrn > 0, qrn, torch.ones_like(qrn)), torch.ones_like(qrn))
            pr1 = qr * scr[:, None]
            pn, pt, pr = pn1, pt1, pr1
            vv, ww = body(pn, pt, pr)
        x1 = x + h * vv
        # geometry forces (impulse on the plane / dt)
        F = torch.zeros((len(self.planes), 3), dtype=torch.float64)
        if ng_c:
            F = F.index_add(0, torch.as_tensor(gg), -(pn[nb:, None] * n[nb:] + pt[nb:]) / h)
        warm1 = {(int(kk[c, 0]), int(kk[c, 1])): torch.cat([pn[c:c + 1], pt[c], pr[c]]) for c in range(nc)}
        plane_pos1 = [pp + h * torch.tensor(pl.v, dtype=torch.float64) for pp, pl in zip(plane_pos, self.planes)]
        return x1, vv, ww, warm1, F, plane_pos1

    def run(self, x, v, w, theta, steps, weights):
        """J = sum over steps of sum_g weights[g] . F_g; returns (J, final x)."""
        x = torch.as_tensor(x, dtype=torch.float64)
        v = torch.as_tensor(v, dtype=torch.float64)
        w = torch.as_tensor(w, dtype=torch.float64)
        W = torch.as_tensor(weights, dtype=torch.float64).reshape(len(self.planes), 3)
        warm = {}
        pp = [torch.tensor(pl.c, dtype=torch.float64) for pl in self.planes]
        J = torch.zeros((), dtype=torch.float64)
        for _ in range(steps):
            x, v, w, warm, F, pp = self.step(x, v, w, theta, warm, pp)
            J = J + (W * F).sum()
        return J, x, v, w


def gradient(params, x, r, v, w, planes, theta, steps, weights, ids=None):
    """(J, dJ/d(kn_scale, mu_t, mu_r)) by autograd through the FP64 steps."""
    ids = np.arange(len(r), dtype=np.int32) if ids is None else ids
    st = TorchStepper(params, r, ids, planes)
    th = [torch.tensor(float(t), dtype=torch.float64, requires_grad=True) for t in theta]
    J, *_ = st.run(x, v, w, th, steps, weights)
    if J.requires_grad:   # no contact in any step: J does not depend on theta
        J.backward()
    return float(J.detach()), np.array([float(t.grad) if t.grad is not None else 0.0 for t in th])
