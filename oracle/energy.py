"""The incremental potential of Eq. (ipc_energy) (oracle, FP64).

    E(x) = 1/2 (x - xhat)^T M (x - xhat) + h^2 Psi(x)
           + kappa * sum_{k in C} b(d_k(x)) + D(x)

  * inertia with the lumped mass M (Eq. varopt);
  * Psi: compressible Neo-Hookean per tet,
        Psi(F) = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2   (times the
        rest volume), +inf when J <= 0;
  * b: the C^2 log barrier b(d) = -(d - dhat)^2 ln(d / dhat) for d < dhat,
        0 otherwise, over point-triangle and edge-edge pairs between the gel
        surface and the rigid indenter; d is the unsigned Euclidean distance;
        an edge-edge term is multiplied by IPC's parallel-edge mollifier
        m(c), c = |e_gel x e_ind|^2 (the distance between two edges has a
        kink where they turn parallel, and the barrier pushes pressed edges
        towards exactly that configuration);
  * D: lagged friction of Eq. (friction_energy) with the mollifier of
        Eq. (friction_mollifier).

Gradients are the textbook formulas (first Piola-Kirchhoff stress, envelope
theorem for distances). Diagonal 3x3 Hessian blocks feed the block-Jacobi
preconditioner: exact for elasticity (with the curvature coefficient clamped
at zero), Gauss-Newton for the barrier, exact for the lagged friction.
Directional derivatives along a line are taken with ``oracle.taylor``.

Pair types (i = gel primitive, j = indenter primitive):
  0: gel vertex i        vs indenter triangle j
  1: gel surface tri i   vs indenter vertex j
  2: gel surface edge i  vs indenter edge j
"""
from __future__ import annotations

import numpy as np

from . import taylor as T

INF = float("inf")

# ---------------------------------------------------------------------------
# elasticity


def _det3(F):
    return (F[..., 0, 0] * (F[..., 1, 1] * F[..., 2, 2] - F[..., 1, 2] * F[..., 2, 1])
            - F[..., 0, 1] * (F[..., 1, 0] * F[..., 2, 2] - F[..., 1, 2] * F[..., 2, 0])
            + F[..., 0, 2] * (F[..., 1, 0] * F[..., 2, 1] - F[..., 1, 1] * F[..., 2, 0]))


def deformation_gradient(x, pad):
    """F = Ds Dm^-1 with Ds = [x1-x0, x2-x0, x3-x0] per tet."""
    t = pad.tets
    Ds = np.stack([x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]], x[t[:, 3]] - x[t[:, 0]]], axis=2)
    return Ds @ pad.Dm_inv


def neo_hookean_density(F, mu, lam):
    """Psi(F) per tet (generic over ndarray / Jet); +inf where J <= 0 for
    plain arrays."""
    J = _det3(F)
    I1 = (F * F).sum(axis=-1).sum(axis=-1)
    if isinstance(J, T.Jet):
        lnJ = T.log(J)
        return 0.5 * mu * (I1 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ
    with np.errstate(invalid="ignore", divide="ignore"):
        lnJ = np.log(J)
        psi = 0.5 * mu * (I1 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ
    return np.where(J > 0, psi, INF)


def first_piola(F, mu, lam):
    """P(F) = mu (F - F^-T) + lam ln J F^-T."""
    J = np.linalg.det(F)
    FinvT = np.swapaxes(np.linalg.inv(F), -1, -2)
    return mu * (F - FinvT) + lam * np.log(J)[:, None, None] * FinvT


def shape_vectors(Dm_inv):
    """b_i = dF/dx_i direction per corner: rows of Dm^-1 for corners 1..3,
    minus their sum for corner 0. Returns [T, 4, 3]."""
    rows = Dm_inv                                     # rows b_1, b_2, b_3
    b0 = -rows.sum(axis=1)
    return np.concatenate([b0[:, None, :], rows], axis=1)


def elastic(x, pad, blocks=True):
    """h^2 * sum_t V_t Psi(F_t), its gradient [V, 3] and (optionally) the
    diagonal 3x3 blocks [V, 3, 3] of its Hessian.

    Diagonal block of corner i (derived from dP = mu dF + (mu - lam ln J)
    F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T with dF = delta b_i^T):
        K_ii = h^2 V [mu |b_i|^2 I + (mu + lam (1 - ln J)) c_i c_i^T],
        c_i = F^-T b_i; the c c^T coefficient is clamped at 0 so that the
    block is positive semi-definite (preconditioner only)."""
    h2 = pad.h * pad.h
    F = deformation_gradient(x, pad)
    J = np.linalg.det(F)
    nV = x.shape[0]
    if np.any(J <= 0):
        return INF, None, None
    psi = neo_hookean_density(F, pad.mu, pad.lam)
    E = h2 * float(np.sum(pad.vol * psi))
    P = first_piola(F, pad.mu, pad.lam)
    H = pad.vol[:, None, None] * (P @ np.swapaxes(pad.Dm_inv, 1, 2))   # dE/dDs
    f = np.zeros((pad.tets.shape[0], 4, 3))
    f[:, 1:, :] = np.swapaxes(H, 1, 2)                 # column i of H is corner i+1
    f[:, 0, :] = -f[:, 1:, :].sum(axis=1)
    g = np.zeros((nV, 3))
    np.add.at(g, pad.tets.ravel(), h2 * f.reshape(-1, 3))
    if not blocks:
        return E, g, None
    b = shape_vectors(pad.Dm_inv)                      # [T, 4, 3]
    FinvT = np.swapaxes(np.linalg.inv(F), 1, 2)
    c = np.einsum("tij,tkj->tki", FinvT, b)            # c_k = F^-T b_k
    coef = np.maximum(pad.mu + pad.lam * (1.0 - np.log(J)), 0.0)
    bb = (b * b).sum(axis=2)                           # |b_k|^2
    K = (pad.mu * bb)[:, :, None, None] * np.eye(3)[None, None] \
        + coef[:, None, None, None] * np.einsum("tki,tkj->tkij", c, c)
    K *= (h2 * pad.vol)[:, None, None, None]
    blk = np.zeros((nV, 3, 3))
    np.add.at(blk, pad.tets.ravel(), K.reshape(-1, 3, 3))
    return E, g, blk


def elastic_line(x, p, pad):
    """Jet of the elastic term along x + t p: (E, g^T p, p^T H p)."""
    xl = T.line(x, p)
    t = pad.tets
    cols = [xl[t[:, k]] - xl[t[:, 0]] for k in (1, 2, 3)]     # [T, 3] each, column k of Ds
    B = pad.Dm_inv
    # F_ab = sum_k Ds_ak B_kb
    F_rows = []
    for a in range(3):
        row = []
        for bcol in range(3):
            acc = cols[0][:, a] * B[:, 0, bcol] + cols[1][:, a] * B[:, 1, bcol] + cols[2][:, a] * B[:, 2, bcol]
            row.append(acc)
        F_rows.append(row)
    Fv = np.stack([np.stack([F_rows[a][b].v for b in range(3)], -1) for a in range(3)], -2)
    Fd = np.stack([np.stack([F_rows[a][b].d for b in range(3)], -1) for a in range(3)], -2)
    Fdd = np.stack([np.stack([F_rows[a][b].dd for b in range(3)], -1) for a in range(3)], -2)
    psi = neo_hookean_density(T.Jet(Fv, Fd, Fdd), pad.mu, pad.lam)
    h2 = pad.h * pad.h
    return (psi * (h2 * pad.vol)).sum()


# ---------------------------------------------------------------------------
# inertia


def inertia(x, xhat, pad):
    """1/2 (x - xhat)^T M (x - xhat), gradient M (x - xhat), blocks m_i I."""
    r = x - xhat
    E = 0.5 * float(np.sum(pad.mass[:, None] * r * r))
    g = pad.mass[:, None] * r
    blk = pad.mass[:, None, None] * np.eye(3)[None]
    return E, g, blk


def inertia_line(x, p, xhat, pad):
    r = T.line(x - xhat, p)
    return (r * r * (0.5 * pad.mass[:, None])).sum()


# ---------------------------------------------------------------------------
# distances (generic over ndarray / Jet); weights describe r = sum_s w_s v_s


def point_segment(P, A, B):
    e = B - A
    t = T.clip01(T.dot(P - A, e) / T.dot(e, e))
    r = P - (A + e * T.expand(t))
    return T.sqrt(T.dot(r, r)), t


def point_triangle(P, A, B, C):
    """Unsigned distance from point P to triangle ABC and the barycentric
    coordinates (values) of the closest point: face interior when the
    projection lies inside, otherwise the nearest edge (endpoints included
    by clamping)."""
    v0, v1, v2 = B - A, C - A, P - A
    d00, d01, d11 = T.dot(v0, v0), T.dot(v0, v1), T.dot(v1, v1)
    d20, d21 = T.dot(v2, v0), T.dot(v2, v1)
    with np.errstate(divide="ignore", invalid="ignore"):
        den = d00 * d11 - d01 * d01
        l1 = (d11 * d20 - d01 * d21) / den
        l2 = (d00 * d21 - d01 * d20) / den
        l0 = 1.0 - l1 - l2
        inside = (T.val(l0) >= 0) & (T.val(l1) >= 0) & (T.val(l2) >= 0)
        n = T.cross(v0, v1)
        dface = T.absolute(T.dot(v2, n)) / T.sqrt(T.dot(n, n))
    dab, tab = point_segment(P, A, B)
    dbc, tbc = point_segment(P, B, C)
    dca, tca = point_segment(P, C, A)
    cand = np.stack([np.where(inside, T.val(dface), INF), T.val(dab), T.val(dbc), T.val(dca)])
    k = np.argmin(cand, axis=0)
    d = T.where(k == 0, dface, T.where(k == 1, dab, T.where(k == 2, dbc, dca)))
    L0, L1, L2 = T.val(l0), T.val(l1), T.val(l2)
    ta, tb, tc = T.val(tab), T.val(tbc), T.val(tca)
    bary = np.stack([
        np.select([k == 0, k == 1, k == 2], [L0, 1 - ta, 0 * ta], tc),
        np.select([k == 0, k == 1, k == 2], [L1, ta, 1 - tb], 0 * tc),
        np.select([k == 0, k == 1, k == 2], [L2, 0 * ta, tb], 1 - tc)], axis=-1)
    return d, bary


def segment_segment(P0, P1, Q0, Q1):
    """Unsigned distance between segments P0P1 and Q0Q1 and the parameters
    (s on P, t on Q, values) of the closest points: both interior when the
    unconstrained line-line solution lies in [0,1]^2 and the lines are not
    parallel, otherwise the best endpoint-to-segment distance."""
    u, v, w = P1 - P0, Q1 - Q0, P0 - Q0
    a, b, c = T.dot(u, u), T.dot(u, v), T.dot(v, v)
    dd, e = T.dot(u, w), T.dot(v, w)
    with np.errstate(divide="ignore", invalid="ignore"):
        D = a * c - b * b
        s = (b * e - c * dd) / D
        t = (a * e - b * dd) / D
        valid = (T.val(D) > 1e-12 * T.val(a) * T.val(c)) & (T.val(s) >= 0) & (T.val(s) <= 1) \
            & (T.val(t) >= 0) & (T.val(t) <= 1)
        r = w + u * T.expand(s) - v * T.expand(t)
        dint = T.sqrt(T.dot(r, r))
    d0, t0 = point_segment(P0, Q0, Q1)
    d1, t1 = point_segment(P1, Q0, Q1)
    d2, t2 = point_segment(Q0, P0, P1)
    d3, t3 = point_segment(Q1, P0, P1)
    cand = np.stack([np.where(valid, T.val(dint), INF), T.val(d0), T.val(d1), T.val(d2), T.val(d3)])
    k = np.argmin(cand, axis=0)
    d = T.where(k == 0, dint, T.where(k == 1, d0, T.where(k == 2, d1, T.where(k == 3, d2, d3))))
    S, Tt = T.val(s), T.val(t)
    a0, a1, a2, a3 = T.val(t0), T.val(t1), T.val(t2), T.val(t3)
    sp = np.select([k == 0, k == 1, k == 2, k == 3], [S, 0 * S, 1 + 0 * S, a2], a3)
    tq = np.select([k == 0, k == 1, k == 2, k == 3], [Tt, a0, a1, 0 * S], 1 + 0 * S)
    return d, sp, tq


def pair_geometry(pairs, x, y, pad, ind):
    """Per pair: the 4 vertex positions (generic) in slot order, the gel
    vertex id of each slot (-1 for indenter slots) and the indenter vertex id
    of each slot (-1 for gel slots).

    Slot layouts: type 0 [gel v, ind tri a, b, c]; type 1 [gel tri a, b, c,
    ind v]; type 2 [gel edge a, b, ind edge a, b]."""
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 3)
    n = pairs.shape[0]
    gid = -np.ones((n, 4), dtype=np.int64)
    iid = -np.ones((n, 4), dtype=np.int64)
    ty, i, j = pairs[:, 0], pairs[:, 1], pairs[:, 2]
    m0, m1, m2 = ty == 0, ty == 1, ty == 2
    gid[m0, 0] = i[m0]
    iid[m0, 1:] = ind.tris[j[m0]]
    gid[m1, :3] = pad.surf_tris[i[m1]]
    iid[m1, 3] = j[m1]
    gid[m2, :2] = pad.surf_edges[i[m2]]
    iid[m2, 2:] = ind.edges[j[m2]]
    return ty, gid, iid


def _slot_positions(gid, iid, x, y):
    """Positions [n, 4, 3] (generic): gel slots from x, indenter slots from y."""
    xv = T.val(x)
    if isinstance(x, T.Jet):
        Pv = np.zeros(gid.shape + (3,))
        Pd = np.zeros(gid.shape + (3,))
        gm = gid >= 0
        Pv[gm] = x.v[gid[gm]]
        Pd[gm] = x.d[gid[gm]]
        Pv[~gm] = y[iid[~gm]]
        return T.Jet(Pv, Pd)
    P = np.zeros(gid.shape + (3,))
    gm = gid >= 0
    P[gm] = xv[gid[gm]]
    P[~gm] = y[iid[~gm]]
    return P


def distances(pairs, x, y, pad, ind):
    """Distances of the candidate pairs. Returns (d, w [n, 4], slots
    (ty, gid, iid)) where r = sum_s w_s v_s points from the indenter to the
    gel (gel weights >= 0, indenter weights <= 0, each side summing to 1).
    With x a Jet, d is a Jet and w holds values."""
    ty, gid, iid = pair_geometry(pairs, x, y, pad, ind)
    P = _slot_positions(gid, iid, x, y)
    d, w = slot_distances(ty, P)
    return d, w, (ty, gid, iid)


def slot_distances(ty, P):
    """Distance and slot weights from slot positions P [n, 4, 3] (generic)."""
    n = ty.shape[0]
    if n == 0:
        return (T.Jet(np.zeros(0)) if isinstance(P, T.Jet) else np.zeros(0)), np.zeros((0, 4))
    dist = T.Jet(np.zeros(n)) if isinstance(P, T.Jet) else np.zeros(n)
    w = np.zeros((n, 4))
    for typ in (0, 1, 2):
        m = np.nonzero(ty == typ)[0]
        if m.size == 0:
            continue
        Q = P[m]
        if typ == 0:
            d, bary = point_triangle(Q[:, 0], Q[:, 1], Q[:, 2], Q[:, 3])
            w[m] = np.concatenate([np.ones((m.size, 1)), -bary], axis=1)
        elif typ == 1:
            d, bary = point_triangle(Q[:, 3], Q[:, 0], Q[:, 1], Q[:, 2])
            w[m] = np.concatenate([bary, -np.ones((m.size, 1))], axis=1)
        else:
            d, s, t = segment_segment(Q[:, 0], Q[:, 1], Q[:, 2], Q[:, 3])
            w[m] = np.stack([1 - s, s, -(1 - t), -t], axis=1)
        if isinstance(dist, T.Jet):
            dist.v[m], dist.d[m], dist.dd[m] = d.v, d.d, d.dd
        else:
            dist[m] = d
    return dist, w


# ---------------------------------------------------------------------------
# barrier


def barrier(d, dhat):
    """b(d) = -(d - dhat)^2 ln(d / dhat) for 0 < d < dhat, else 0 (generic)."""
    if isinstance(d, T.Jet):
        inner = -((d - dhat) * (d - dhat)) * T.log(d / dhat)
        return T.where(d.v < dhat, inner, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(d < dhat, -(d - dhat) ** 2 * np.log(d / dhat), 0.0)


def barrier_d1(d, dhat):
    """b'(d) = -2 (d - dhat) ln(d/dhat) - (d - dhat)^2 / d (0 beyond dhat)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(d < dhat, -2.0 * (d - dhat) * np.log(d / dhat) - (d - dhat) ** 2 / d, 0.0)


def barrier_d2(d, dhat):
    """b''(d) = -2 ln(d/dhat) - 4 (d - dhat)/d + (d - dhat)^2 / d^2."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(d < dhat, -2.0 * np.log(d / dhat) - 4.0 * (d - dhat) / d + (d - dhat) ** 2 / d ** 2, 0.0)


# ---------------------------------------------------------------------------
# parallel-edge mollifier of the edge-edge terms (IPC, Li et al. 2020)

EE_MOLLIFIER_REL = 1e-3


def ee_mollifier_eps(ty, gid, iid, pad, ind):
    """Mollifier threshold of each pair: eps_x = 1e-3 |gel edge|^2
    |indenter edge|^2 with rest lengths for an edge-edge pair (type 2), 0
    (no mollifier) for the point-triangle types."""
    eps = np.zeros(len(ty))
    m = ty == 2
    if np.any(m):
        a = pad.rest[gid[m, 1]] - pad.rest[gid[m, 0]]
        b = ind.verts[iid[m, 3]] - ind.verts[iid[m, 2]]
        eps[m] = EE_MOLLIFIER_REL * np.einsum("nc,nc->n", a, a) * np.einsum("nc,nc->n", b, b)
    return eps


def edge_cross_sq(P):
    """c = |(P1 - P0) x (Q1 - Q0)|^2 of slot positions [P0, P1, Q0, Q1]
    (generic)."""
    w = T.cross(P[:, 1] - P[:, 0], P[:, 3] - P[:, 2])
    return T.dot(w, w)


def edge_cross_sq_grad(P):
    """c and dc/d(slot position) [n, 4, 3] (values): with u = P1 - P0,
    v = Q1 - Q0, w = u x v, dc = 2 (v x w).du + 2 (w x u).dv."""
    u, v = P[:, 1] - P[:, 0], P[:, 3] - P[:, 2]
    w = np.cross(u, v)
    gu, gv = 2.0 * np.cross(v, w), 2.0 * np.cross(w, u)
    return np.einsum("nc,nc->n", w, w), np.stack([-gu, gu, -gv, gv], axis=1)


def ee_mollifier(c, eps):
    """m(c) = (2 - c/eps) c/eps for c < eps, else 1 (generic in c); a pair
    with eps = 0 gets 1. C^1 at c = eps, m(0) = 0."""
    on = T.val(c) < eps
    inv = np.where(eps > 0, 1.0 / np.where(eps > 0, eps, 1.0), 0.0)
    q = c * inv
    return T.where(on, (2.0 - q) * q, 1.0)


def ee_mollifier_d1(c, eps):
    """m'(c) = 2/eps (1 - c/eps) for c < eps, else 0 (values)."""
    inv = np.where(eps > 0, 1.0 / np.where(eps > 0, eps, 1.0), 0.0)
    return np.where(c < eps, 2.0 * inv * (1.0 - c * inv), 0.0)


def pair_barrier(ty, P, eps, dhat):
    """Per pair m(c) b(d) from slot positions P [n, 4, 3] (generic: with P
    a Jet along a line the result carries the line derivatives)."""
    d, _ = slot_distances(ty, P)
    return ee_mollifier(edge_cross_sq(P), eps) * barrier(d, dhat)


def contact(pairs, x, y, pad, ind):
    """kappa * sum m(c_k) b(d_k), its gradient on gel vertices and
    Gauss-Newton diagonal blocks kappa m(c) b''(d) w_s^2 r^ r^T (the
    mollifier's own derivatives left out of the blocks). Returns (E, g,
    blk, dmin)."""
    nV = x.shape[0]
    g = np.zeros((nV, 3))
    blk = np.zeros((nV, 3, 3))
    if len(pairs) == 0:
        return 0.0, g, blk, INF
    d, w, (ty, gid, iid) = distances(pairs, x, y, pad, ind)
    if np.any(d <= 0):
        return INF, None, None, float(d.min())
    P = _slot_positions(gid, iid, x, y)
    r = np.einsum("ns,nsk->nk", w, P)
    rhat = r / d[:, None]
    dh = pad.dhat
    eps = ee_mollifier_eps(ty, gid, iid, pad, ind)
    c, gc = edge_cross_sq_grad(P)
    mv, m1 = ee_mollifier(c, eps), ee_mollifier_d1(c, eps)
    bv = barrier(d, dh)
    E = pad.kappa * float(np.sum(mv * bv))
    b1 = pad.kappa * mv * barrier_d1(d, dh)
    b2 = pad.kappa * mv * barrier_d2(d, dh)
    cb = pad.kappa * m1 * bv
    for s in range(4):
        m = gid[:, s] >= 0
        np.add.at(g, gid[m, s], (b1[m] * w[m, s])[:, None] * rhat[m] + cb[m][:, None] * gc[m, s])
        np.add.at(blk, gid[m, s], (b2[m] * w[m, s] ** 2)[:, None, None] * np.einsum("ni,nj->nij", rhat[m], rhat[m]))
    return E, g, blk, float(d.min())


def contact_line(pairs, x, p, y, pad, ind):
    if len(pairs) == 0:
        return T.Jet(0.0)
    ty, gid, iid = pair_geometry(pairs, x, y, pad, ind)
    P = _slot_positions(gid, iid, T.line(x, p), y)
    eps = ee_mollifier_eps(ty, gid, iid, pad, ind)
    return pair_barrier(ty, P, eps, pad.dhat).sum() * pad.kappa


# ---------------------------------------------------------------------------
# lagged friction


def mollifier(s, eps):
    """f(s) of Eq. (friction_mollifier)."""
    return np.where(s < eps, -s ** 3 / (3 * eps * eps) + s * s / eps + eps / 3, s)


def mollifier_d1_over_s(s, eps):
    """f'(s) / s (finite at s = 0)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(s < eps, -s / (eps * eps) + 2.0 / eps, 1.0 / s)


def friction_lag(pairs, x_t, y_t, pad, ind):
    """Lag data from the state at the start of the frame: every candidate
    pair with d < dhat contributes lambda_n = -kappa m(c) b'(d) (the normal
    force of its mollified barrier), the normal r^ and
    the closest-point weights (gel slots w >= 0, indenter slots w <= 0)."""
    empty = dict(gid=np.zeros((0, 4), np.int64), iid=np.zeros((0, 4), np.int64), w=np.zeros((0, 4)),
                 n=np.zeros((0, 3)), lam=np.zeros(0))
    if len(pairs) == 0 or pad.mu_f == 0.0:
        return empty
    d, w, (ty, gid, iid) = distances(pairs, x_t, y_t, pad, ind)
    act = d < pad.dhat
    if not np.any(act):
        return empty
    P = _slot_positions(gid[act], iid[act], x_t, y_t)
    r = np.einsum("ns,nsk->nk", w[act], P)
    mv = ee_mollifier(edge_cross_sq(P), ee_mollifier_eps(ty[act], gid[act], iid[act], pad, ind))
    return dict(gid=gid[act], iid=iid[act], w=w[act], n=r / d[act][:, None],
                lam=-pad.kappa * mv * barrier_d1(d[act], pad.dhat))


def _friction_disp(lag, x, x_t, y, y_t):
    """Relative displacement of the lagged closest points since the frame
    start: sum_s w_s (v_s - v_s^t) (generic in x)."""
    gid, iid, w = lag["gid"], lag["iid"], lag["w"]
    n = gid.shape[0]
    dy = np.zeros((n, 3))
    for s in range(4):
        m = iid[:, s] >= 0
        dy[m] += w[m, s][:, None] * (y[iid[m, s]] - y_t[iid[m, s]])
    if isinstance(x, T.Jet):
        acc = T.Jet(dy)
        for s in range(4):
            m = gid[:, s] >= 0
            col = T.Jet(np.zeros((n, 3)))
            col.v[m] = x.v[gid[m, s]] - x_t[gid[m, s]]
            col.d[m] = x.d[gid[m, s]]
            acc = acc + col * w[:, s][:, None]
        return acc
    dx = dy.copy()
    for s in range(4):
        m = gid[:, s] >= 0
        dx[m] += w[m, s][:, None] * (x[gid[m, s]] - x_t[gid[m, s]])
    return dx


def friction(lag, x, x_t, y, y_t, pad):
    """D = mu_f sum lambda_n f(|Pi Delta|), Pi = I - n n^T; gradient and the
    (positive semi-definite) exact diagonal blocks
        mu lam w^2 [f'(s)/s Pi - c(s) u u^T],  u = Pi Delta / s,
        c(s) = s/eps^2 (s < eps) or 1/s (s >= eps)."""
    nV = x.shape[0]
    g = np.zeros((nV, 3))
    blk = np.zeros((nV, 3, 3))
    if lag["lam"].size == 0 or pad.mu_f == 0.0:
        return 0.0, g, blk
    eps = pad.eps_v
    nrm = lag["n"]
    Pi = np.eye(3)[None] - np.einsum("ni,nj->nij", nrm, nrm)
    D = _friction_disp(lag, x, x_t, y, y_t)
    tD = np.einsum("nij,nj->ni", Pi, D)
    s = np.linalg.norm(tD, axis=1)
    c = pad.mu_f * lag["lam"]
    E = float(np.sum(c * mollifier(s, eps)))
    f1s = mollifier_d1_over_s(s, eps)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.where(s[:, None] > 0, tD / s[:, None], 0.0)
    cs = np.where(s < eps, s / (eps * eps), np.where(s > 0, 1.0 / np.maximum(s, 1e-300), 0.0))
    Hn = f1s[:, None, None] * Pi - cs[:, None, None] * np.einsum("ni,nj->nij", u, u)
    gid, w = lag["gid"], lag["w"]
    for sl in range(4):
        m = gid[:, sl] >= 0
        np.add.at(g, gid[m, sl], (c[m] * f1s[m] * w[m, sl])[:, None] * tD[m])
        np.add.at(blk, gid[m, sl], (c[m] * w[m, sl] ** 2)[:, None, None] * Hn[m])
    return E, g, blk


def friction_line(lag, x, p, x_t, y, y_t, pad):
    if lag["lam"].size == 0 or pad.mu_f == 0.0:
        return T.Jet(0.0)
    eps = pad.eps_v
    nrm = lag["n"]
    D = _friction_disp(lag, T.line(x, p), x_t, y, y_t)
    # tangential part Pi D = D - n (n . D)
    nd = T.dot(D, nrm)
    tD = D - nrm * T.expand(nd)
    q = T.dot(tD, tD)
    small = q.v < (1e-12 * eps) ** 2
    qs = T.Jet(np.where(small, 1.0, q.v), np.where(small, 0.0, q.d), np.where(small, 0.0, q.dd))
    s = T.sqrt(qs)
    f_in = -(s * s * s) / (3 * eps * eps) + qs / eps + eps / 3
    f = T.where(s.v < eps, f_in, s)
    f = T.where(small, q / eps + eps / 3, f)          # quadratic limit at s -> 0
    return (f * (pad.mu_f * lag["lam"])).sum()


# ---------------------------------------------------------------------------
# totals


class Frame:
    """Everything fixed during one frame solve (besides x and s)."""

    def __init__(self, pad, ind, x_t, xhat, y_t, y_next, lag):
        self.pad, self.ind = pad, ind
        self.x_t, self.xhat = x_t, xhat
        self.y_t, self.y_next = y_t, y_next
        self.lag = lag

    def y(self, s):
        """Indenter vertices at path parameter s (per-vertex linear path)."""
        return (1.0 - s) * self.y_t + s * self.y_next


def total(fr, x, s, pairs, blocks=True):
    """E(x), gradient and diagonal blocks at path parameter s."""
    pad = fr.pad
    y = fr.y(s)
    Ei, gi, bi = inertia(x, fr.xhat, pad)
    Ee, ge, be = elastic(x, pad, blocks=True)
    if not np.isfinite(Ee):
        return INF, None, None
    Ec, gc, bc, _ = contact(pairs, x, y, pad, fr.ind)
    if not np.isfinite(Ec):
        return INF, None, None
    Ef, gf, bf = friction(fr.lag, x, fr.x_t, y, fr.y_t, pad)
    g = gi + ge + gc + gf
    blk = bi + be + bc + bf
    g[~pad.free] = 0.0
    return Ei + Ee + Ec + Ef, g, blk


def total_line(fr, x, p, s, pairs):
    """Jet of E(x + t p) at t = 0: (E, g^T p, p^T H p)."""
    pad = fr.pad
    y = fr.y(s)
    return (inertia_line(x, p, fr.xhat, pad) + elastic_line(x, p, pad)
            + contact_line(pairs, x, p, y, pad, fr.ind)
            + friction_line(fr.lag, x, p, fr.x_t, y, fr.y_t, pad))


def energy_only(fr, x, s, pairs):
    pad = fr.pad
    y = fr.y(s)
    Ei, _, _ = inertia(x, fr.xhat, pad)
    F = deformation_gradient(x, pad)
    psi = neo_hookean_density(F, pad.mu, pad.lam)
    if not np.all(np.isfinite(psi)):
        return INF
    Ee = pad.h * pad.h * float(np.sum(pad.vol * psi))
    if len(pairs):
        d, _, (ty, gid, iid) = distances(pairs, x, y, pad, fr.ind)
        if np.any(d <= 0):
            return INF
        P = _slot_positions(gid, iid, x, y)
        mv = ee_mollifier(edge_cross_sq(P), ee_mollifier_eps(ty, gid, iid, pad, fr.ind))
        Ec = pad.kappa * float(np.sum(mv * barrier(d, pad.dhat)))
    else:
        Ec = 0.0
    Ef, _, _ = friction(fr.lag, x, fr.x_t, y, fr.y_t, pad)
    return Ei + Ee + Ec + Ef
