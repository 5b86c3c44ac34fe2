"""Newton certification of a PNCG end point and the exact Hessian (oracle).

The assembled Hessian H = M + h^2 grad^2 Psi + kappa sum grad^2 b + grad^2 D
(Supp. A) over the free DOFs:
  * elastic: per tet, the exact 12x12 block from the stress differential
        dP = mu dF + (mu - lam ln J) F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T;
  * barrier: per pair, the exact Hessian in the pair's gel DOFs by
        polarisation of second directional derivatives (oracle.taylor);
  * friction: per lagged pair, mu lam w_s w_s' [f'(s)/s Pi - c(s) u u^T].
Newton's method from the PNCG result (full steps bounded by the CCD rule,
Armijo in remainder form) then gives the frame's minimiser to near machine
precision; the distance between the two is the PNCG end point's error.
"""
from __future__ import annotations

import numpy as np

from . import energy as En
from . import solver as SV
from . import taylor as T


def elastic_hessian_blocks(x, pad):
    """Exact per-tet Hessian [T, 4, 3, 4, 3] (times h^2 V)."""
    F = En.deformation_gradient(x, pad)
    J = np.linalg.det(F)
    Finv = np.linalg.inv(F)
    FinvT = np.swapaxes(Finv, 1, 2)
    lnJ = np.log(J)
    b = En.shape_vectors(pad.Dm_inv)
    nT = F.shape[0]
    H = np.zeros((nT, 4, 3, 4, 3))
    for j in range(4):
        for c in range(3):
            dF = np.zeros((nT, 3, 3))
            dF[:, c, :] = b[:, j, :]                               # e_c b_j^T
            dP = (pad.mu * dF
                  + (pad.mu - pad.lam * lnJ)[:, None, None] * (FinvT @ np.swapaxes(dF, 1, 2) @ FinvT)
                  + (pad.lam * np.einsum("tii->t", Finv @ dF))[:, None, None] * FinvT)
            H[:, :, :, j, c] = np.einsum("tab,tib->tia", dP, b)     # dP b_i
    return H * (pad.h * pad.h * pad.vol)[:, None, None, None, None]


def _pair_hessians(fr, x, s, pairs):
    """Exact barrier Hessian per pair over its 4 slots [n, 4, 3, 4, 3]
    (indenter slots are zero), by polarisation of Jet second derivatives."""
    pad = fr.pad
    y = fr.y(s)
    ty, gid, iid = En.pair_geometry(pairs, x, y, pad, fr.ind)
    P = En._slot_positions(gid, iid, x, y)
    n = len(ty)
    gm = gid >= 0
    dofs = [(sl, c) for sl in range(4) for c in range(3)]
    Q = {}

    eps = En.ee_mollifier_eps(ty, gid, iid, pad, fr.ind)

    def q(dirs):
        return pad.kappa * En.pair_barrier(ty, T.Jet(P, dirs), eps, pad.dhat).dd

    diag = []
    for k, (sl, c) in enumerate(dofs):
        dv = np.zeros((n, 4, 3))
        dv[:, sl, c] = gm[:, sl]
        diag.append(q(dv))
    H = np.zeros((n, 4, 3, 4, 3))
    for a, (s1, c1) in enumerate(dofs):
        H[:, s1, c1, s1, c1] = diag[a]
        for b_, (s2, c2) in enumerate(dofs[a + 1:], start=a + 1):
            dv = np.zeros((n, 4, 3))
            dv[:, s1, c1] = gm[:, s1]
            dv[:, s2, c2] += gm[:, s2]
            v = 0.5 * (q(dv) - diag[a] - diag[b_])
            H[:, s1, c1, s2, c2] = v
            H[:, s2, c2, s1, c1] = v
    return gid, H


def assemble(fr, x, s, pairs):
    """Dense exact Hessian [3V, 3V] (all DOFs; Dirichlet rows untouched)."""
    pad = fr.pad
    nV = x.shape[0]
    H = np.zeros((3 * nV, 3 * nV))
    idx = np.arange(3 * nV)
    H[idx, idx] += np.repeat(pad.mass, 3)
    He = elastic_hessian_blocks(x, pad)
    t = pad.tets
    for i in range(4):
        for j in range(4):
            for a in range(3):
                for c in range(3):
                    np.add.at(H, (3 * t[:, i] + a, 3 * t[:, j] + c), He[:, i, a, j, c])
    if len(pairs):
        gid, Hp = _pair_hessians(fr, x, s, pairs)
        for s1 in range(4):
            for s2 in range(4):
                m = (gid[:, s1] >= 0) & (gid[:, s2] >= 0)
                for a in range(3):
                    for c in range(3):
                        np.add.at(H, (3 * gid[m, s1] + a, 3 * gid[m, s2] + c), Hp[m, s1, a, s2, c])
    lag = fr.lag
    if lag["lam"].size and pad.mu_f > 0:
        eps = pad.eps_v
        y = fr.y(s)
        nrm = lag["n"]
        Pi = np.eye(3)[None] - np.einsum("ni,nj->nij", nrm, nrm)
        D = En._friction_disp(lag, x, fr.x_t, y, fr.y_t)
        tD = np.einsum("nij,nj->ni", Pi, D)
        sv = np.linalg.norm(tD, axis=1)
        with np.errstate(divide="ignore", invalid="ignore"):
            u = np.where(sv[:, None] > 0, tD / sv[:, None], 0.0)
        cs = np.where(sv < eps, sv / (eps * eps), np.where(sv > 0, 1.0 / np.maximum(sv, 1e-300), 0.0))
        Hn = En.mollifier_d1_over_s(sv, eps)[:, None, None] * Pi - cs[:, None, None] * np.einsum("ni,nj->nij", u, u)
        c = pad.mu_f * lag["lam"]
        gid, w = lag["gid"], lag["w"]
        for s1 in range(4):
            for s2 in range(4):
                m = (gid[:, s1] >= 0) & (gid[:, s2] >= 0)
                blk = (c[m] * w[m, s1] * w[m, s2])[:, None, None] * Hn[m]
                for a in range(3):
                    for cc in range(3):
                        np.add.at(H, (3 * gid[m, s1] + a, 3 * gid[m, s2] + cc), blk[:, a, cc])
    return H


def newton_polish(fr, x0, s, prm=SV.Params(), max_iter=30, tol_rel=1e-12):
    """Newton iterations from x0 at path parameter s. Returns (x, |g|_inf,
    iterations). Pairs are rebuilt each iteration (full candidate set)."""
    from . import broadphase as BP
    pad = fr.pad
    free = pad.free
    fdof = np.repeat(free, 3)
    x = x0.copy()
    r = pad.dhat * (1.0 + prm.margin_factor)
    it = 0
    for it in range(max_iter):
        pairs = BP.candidates(x, fr.y(s), pad, fr.ind, r)
        E, g, _ = En.total(fr, x, s, pairs)
        gi = float(np.abs(g[free]).max())
        if gi <= tol_rel * pad.g_ref:
            return x, gi, it
        H = assemble(fr, x, s, pairs)
        Hf = H[np.ix_(fdof, fdof)]
        step = np.zeros(3 * x.shape[0])
        step[fdof] = np.linalg.solve(Hf, -g.ravel()[fdof])
        p = step.reshape(-1, 3)
        pn = SV.vnorm_max(p)
        alpha = min(1.0, SV.ccd_bound(fr, x, p, s, pairs, prm.eta), pad.dhat / (2.0 * pn) if pn > 0 else 1.0)
        gTp = float(np.sum(g * p))
        for _ in range(40):
            R = SV.remainder(fr, x, p, alpha, s, pairs)
            if R <= (1.0 - prm.armijo_c) * alpha * (-gTp):
                break
            alpha *= 0.5
        x = x + alpha * p
    pairs = BP.candidates(x, fr.y(s), pad, fr.ind, r)
    _, g, _ = En.total(fr, x, s, pairs)
    return x, float(np.abs(g[free]).max()), it + 1


def certify(pad, ind, state_prev, state_new, prm=SV.Params()):
    """Newton-polish the frame that led from state_prev to state_new and
    return (x_newton, max vertex |x_pncg - x_newton|, |g|_inf at x_newton)."""
    from . import broadphase as BP
    from . import geometry as G
    x_t = state_prev.x
    xhat = x_t + pad.h * state_prev.v
    y_t = G.indenter_world(ind.verts, state_prev.pose)
    y_n = G.indenter_world(ind.verts, state_new.pose)
    cand = BP.candidates(x_t, y_t, pad, ind, pad.dhat * (1.0 + prm.margin_factor))
    lag = En.friction_lag(cand, x_t, y_t, pad, ind)
    fr = En.Frame(pad, ind, x_t, xhat, y_t, y_n, lag)
    xn, gi, _ = newton_polish(fr, state_new.x, 1.0, prm)
    err = float(np.sqrt(((state_new.x - xn) ** 2).sum(axis=1)).max())
    return xn, err, gi
