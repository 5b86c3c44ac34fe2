"""Per-frame PNCG-IPC solve (oracle, FP64), Supp. A.

One frame minimises E of Eq. (ipc_energy) from x^t with xhat = x^t + h v^t
(Eq. varopt) by the Dai-Kou preconditioned nonlinear CG of Eq. (dk_direction)
with the step rule of Eq. (step_size). Readings where the paper is silent:

  * preconditioner: P = (3x3 diagonal blocks of H)^-1 per free vertex
    (block-Jacobi; ``precond="scalar"`` gives the literal diag(H)^-1);
  * step: alpha = min(alpha_upper, alpha_ccd, alpha_bar) with
    alpha_upper = dhat / (2 max_i |p_i|), alpha_ccd = eta * min_k d_k /
    max_{i in gel side of k} |p_i| (eta = 0.9), alpha_bar = -g^T p / p^T H p
    (dropped when p^T H p <= 0); then Armijo backtracking (c = 1e-4, halve
    up to 20 times). The Armijo test E(x + a p) <= E(x) + c a g^T p is
    evaluated in its equivalent remainder form R(a) <= (1 - c) a |g^T p|,
    R(a) = E(x + a p) - E(x) - a g^T p summed element by element.
    ``step="literal"`` is Eq. (step_size) as printed: alpha = min(alpha_upper,
    alpha_bar), no CCD bound and no energy test; a trial state outside E's
    domain (an inverted tet, a closed gap) is still halved;
  * direction restart (beta = 0) when |y^T p| is negligible or the new p
    is not a descent direction; a line search that fails along a conjugate
    direction is retried once along -P g before it counts as failed;
  * stopping: max_i |g_i| (free DOFs) <= tol * g_ref, g_ref = max(h^2 E
    l-bar dhat, max_i |g_i| at the frame's first evaluation after the first
    indenter substep);
  * indenter motion: the indenter vertices move on the straight path
    y(s) = (1 - s) y^t + s y^{t+1}, and the gel moves with them: a substep
    advances s by ds and the gel by ds w, w = xhat - x^t the inertial
    prediction of Eq. varopt (zero on Dirichlet vertices), the same for
    every substep of the frame. ds is at most
    eta * d_k / max_{i in gel(k), j in ind(k)} |w_i - dy_j| for every
    candidate k (dy = y^{t+1} - y^t): along straight motions of both sides
    the points of two primitives approach at most that fast, so no gap
    closes by more than eta of itself. When holding the gel (w = 0 in the
    same bound) allows a longer substep, the substep holds it. ds is halved
    while the advanced state leaves E's domain (an inverted tet). Each
    substep is followed by PNCG to tol_advance (1e-2) relative, the last
    (s = 1) to tol;
  * candidate set: rebuilt whenever the accumulated motion bound since the
    last build would exceed the margin m (= dhat), so pairs outside the set
    stay farther than dhat; an advance moves any gel-indenter point pair
    by at most ds B, B = max_j |dy_j - dy_0| + max_i |w_i - dy_0| (gel
    moving) or max_j |dy_j| (gel held);
  * friction lag (lambda_n, normal, closest-point weights) from x^t with the
    indenter at y^t, once per frame.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import broadphase as BP
from . import energy as En
from . import geometry as G

CONVERGED, MAXITER, NONFINITE, LINESEARCH = 0, 1, 2, 3


@dataclasses.dataclass
class Params:
    tol: float = 1e-6
    tol_advance: float = 1e-2
    max_iter: int = 10000
    eta: float = 0.9
    armijo_c: float = 1e-4
    max_halvings: int = 20
    max_substeps: int = 4000
    margin_factor: float = 1.0        # m = margin_factor * dhat
    precond: str = "block"
    step: str = "bounded"             # "literal": alpha = min(alpha_upper, alpha_bar), no CCD, no Armijo


@dataclasses.dataclass
class State:
    x: np.ndarray        # [V, 3] positions
    v: np.ndarray        # [V, 3] velocities
    pose: np.ndarray     # [6] indenter pose of this state


def rest_state(pad, pose):
    return State(x=pad.rest.copy(), v=np.zeros_like(pad.rest), pose=np.asarray(pose, np.float64).copy())


def precondition(blk, free, mode):
    """P per vertex: inverse of the 3x3 diagonal block (block mode) or of its
    diagonal (scalar mode); zero on Dirichlet vertices."""
    P = np.zeros_like(blk)
    if mode == "block":
        P[free] = np.linalg.inv(blk[free])
    else:
        dg = np.einsum("nii->ni", blk[free])
        P[free] = np.einsum("ni,ij->nij", 1.0 / dg, np.eye(3))
    return P


def apply_P(P, v):
    return np.einsum("nij,nj->ni", P, v)


def vnorm_max(v):
    """max over vertices of the Euclidean norm."""
    return float(np.sqrt((v * v).sum(axis=1)).max()) if v.size else 0.0


def ccd_bound(fr, x, p, s, pairs, eta):
    """eta * min_k d_k / max_{gel slots of k} |p_i| over the candidates."""
    if len(pairs) == 0:
        return np.inf
    d, w, (ty, gid, iid) = En.distances(pairs, x, fr.y(s), fr.pad, fr.ind)
    pn = np.sqrt((p * p).sum(axis=1))
    pk = np.zeros(len(pairs))
    for sl in range(4):
        m = gid[:, sl] >= 0
        pk[m] = np.maximum(pk[m], pn[gid[m, sl]])
    ok = pk > 0
    if not np.any(ok):
        return np.inf
    return float(np.min(eta * d[ok] / pk[ok]))


def dk_beta(g_new, yv, p, P_new):
    """Dai-Kou conjugate parameter of Eq. (dk_direction):
        beta = g^T P y / y^T p - (y^T P y / y^T p) (p^T g / y^T p)
    with g = g_{k+1}, y = g_{k+1} - g_k, p = p_k, P = P_{k+1}; 0 when y^T p
    is negligible (restart)."""
    yp = float(np.sum(yv * p))
    if not (abs(yp) > 1e-300 and abs(yp) > 1e-14 * np.linalg.norm(yv) * np.linalg.norm(p)):
        return 0.0
    Py = apply_P(P_new, yv)
    return float(np.sum(g_new * Py)) / yp - (float(np.sum(yv * Py)) / yp) * (float(np.sum(p * g_new)) / yp)


def relative_motion(fr, pairs, w, dy):
    """Per candidate, max over its gel vertices i and indenter vertices j of
    |w_i - dy_j|: the fastest approach of any point pair of the two
    primitives when the gel moves by w and the indenter by dy."""
    ty, gid, iid = En.pair_geometry(pairs, fr.x_t, fr.y_t, fr.pad, fr.ind)
    out = np.zeros(len(ty))
    for a in range(4):
        for b in range(4):
            m = (gid[:, a] >= 0) & (iid[:, b] >= 0)
            if np.any(m):
                out[m] = np.maximum(out[m], np.linalg.norm(w[gid[m, a]] - dy[iid[m, b]], axis=1))
    return out


def advance_bound(fr, x, s, pairs, w, dy, eta):
    """eta * min_k d_k / (relative motion of k): the largest advance of s
    (gel along w, indenter along dy) that keeps every candidate's gap above
    (1 - eta) of itself."""
    if len(pairs) == 0:
        return np.inf
    d, _, _ = En.distances(pairs, x, fr.y(s), fr.pad, fr.ind)
    rel = relative_motion(fr, pairs, w, dy)
    ok = rel > 0
    return float(np.min(eta * d[ok] / rel[ok])) if np.any(ok) else np.inf


def min_distance(fr, x, s, pairs):
    if len(pairs) == 0:
        return np.inf
    d, _, _ = En.distances(pairs, x, fr.y(s), fr.pad, fr.ind)
    return float(d.min())


def remainder(fr, x, p, alpha, s, pairs):
    """R(alpha) = E(x + alpha p) - E(x) - alpha g^T p, summed per element:
    inertia (exact: alpha^2/2 p^T M p), each tet, each pair, each lagged
    friction pair. +inf when the trial state inverts a tet or closes a gap."""
    pad = fr.pad
    y = fr.y(s)
    xa = x + alpha * p
    R = 0.5 * alpha * alpha * float(np.sum(pad.mass[:, None] * p * p))
    # elasticity
    F0 = En.deformation_gradient(x, pad)
    F1 = En.deformation_gradient(xa, pad)
    if np.any(np.linalg.det(F1) <= 0):
        return np.inf
    t = pad.tets
    Dp = np.stack([p[t[:, 1]] - p[t[:, 0]], p[t[:, 2]] - p[t[:, 0]], p[t[:, 3]] - p[t[:, 0]]], axis=2)
    dF = Dp @ pad.Dm_inv
    P0 = En.first_piola(F0, pad.mu, pad.lam)
    psi0 = En.neo_hookean_density(F0, pad.mu, pad.lam)
    psi1 = En.neo_hookean_density(F1, pad.mu, pad.lam)
    R += pad.h * pad.h * float(np.sum(pad.vol * (psi1 - psi0 - alpha * np.einsum("tij,tij->t", P0, dF))))
    # barrier (edge-edge terms mollified: m(c) b(d))
    if len(pairs):
        d0, w, (ty, gid, iid) = En.distances(pairs, x, y, pad, fr.ind)
        d1, _, _ = En.distances(pairs, xa, y, pad, fr.ind)
        if np.any(d1 <= 0):
            return np.inf
        P = En._slot_positions(gid, iid, x, y)
        P1 = En._slot_positions(gid, iid, xa, y)
        eps = En.ee_mollifier_eps(ty, gid, iid, pad, fr.ind)
        c0, gc = En.edge_cross_sq_grad(P)
        m0, m0d = En.ee_mollifier(c0, eps), En.ee_mollifier_d1(c0, eps)
        m1 = En.ee_mollifier(En.edge_cross_sq(P1), eps)
        r = np.einsum("ns,nsk->nk", w, P)
        rhat = r / d0[:, None]
        pslots = np.zeros(gid.shape + (3,))
        gm = gid >= 0
        pslots[gm] = p[gid[gm]]
        ddot = np.einsum("ns,nsk,nk->n", w * gm, pslots, rhat)       # grad d . p
        cdot = np.einsum("nsk,nsk->n", gc, pslots)                    # grad c . p
        b0 = En.barrier(d0, pad.dhat)
        R += pad.kappa * float(np.sum(m1 * En.barrier(d1, pad.dhat) - m0 * b0
                                      - alpha * (m0 * En.barrier_d1(d0, pad.dhat) * ddot + m0d * cdot * b0)))
    # friction
    lag = fr.lag
    if lag["lam"].size and pad.mu_f > 0:
        eps = pad.eps_v
        nrm = lag["n"]
        Pi = np.eye(3)[None] - np.einsum("ni,nj->nij", nrm, nrm)
        D0 = En._friction_disp(lag, x, fr.x_t, y, fr.y_t)
        D1 = En._friction_disp(lag, xa, fr.x_t, y, fr.y_t)
        tD0 = np.einsum("nij,nj->ni", Pi, D0)
        tD1 = np.einsum("nij,nj->ni", Pi, D1)
        s0, s1 = np.linalg.norm(tD0, axis=1), np.linalg.norm(tD1, axis=1)
        gid, w = lag["gid"], lag["w"]
        pd = np.zeros_like(D0)
        for sl in range(4):
            m = gid[:, sl] >= 0
            pd[m] += w[m, sl][:, None] * p[gid[m, sl]]
        c = pad.mu_f * lag["lam"]
        first = c * En.mollifier_d1_over_s(s0, eps) * np.einsum("ni,ni->n", tD0, pd)
        R += float(np.sum(c * (En.mollifier(s1, eps) - En.mollifier(s0, eps)) - alpha * first))
    return R


@dataclasses.dataclass
class FrameInfo:
    status: int = CONVERGED
    iters: int = 0
    substeps: int = 0
    rebuilds: int = 0
    halvings: int = 0
    grad_inf: float = 0.0
    g_ref: float = 0.0
    min_gap: float = np.inf
    energy_monotone: bool = True


def solve_frame(pad, ind, state, pose_next, prm=Params(), trace=None, lag=None):
    """Advance one frame from ``state`` to the indenter pose ``pose_next``.
    Returns (new State, FrameInfo). ``trace``, if a list, receives per
    iteration (x-step size, energy, |g|_inf). ``lag``, if given, replaces
    the friction lag computed from the frame's start (used to re-solve a
    frame with the lag of another run held fixed)."""
    info = FrameInfo(g_ref=pad.g_ref)
    h, dhat = pad.h, pad.dhat
    margin = prm.margin_factor * dhat
    r_inf = dhat + margin
    x_t = state.x.copy()
    xhat = x_t + h * state.v
    y_t = G.indenter_world(ind.verts, state.pose)
    y_n = G.indenter_world(ind.verts, pose_next)
    cand = BP.candidates(x_t, y_t, pad, ind, r_inf)
    if lag is None:
        lag = En.friction_lag(cand, x_t, y_t, pad, ind)
    fr = En.Frame(pad, ind, x_t, xhat, y_t, y_n, lag)
    dy = y_n - y_t
    free = pad.free
    w_pred = xhat - x_t                 # predicted gel motion over the frame
    w_pred[~free] = 0.0
    held = np.zeros_like(w_pred)
    B_pred = float(np.linalg.norm(dy - dy[0], axis=1).max() + np.linalg.norm(w_pred - dy[0], axis=1).max())
    B_held = float(np.linalg.norm(dy, axis=1).max())
    x = x_t.copy()
    s, M = 0.0, 0.0
    info.min_gap = min_distance(fr, x, s, cand)
    g_ref = None

    def choose(cand, cap):
        # the longer of the two advances (gel moving with the prediction or held)
        dp = min(1.0 - s, advance_bound(fr, x, s, cand, w_pred, dy, prm.eta), cap(B_pred))
        dh = min(1.0 - s, advance_bound(fr, x, s, cand, held, dy, prm.eta), cap(B_held))
        return (dp, w_pred, B_pred) if dp >= dh else (dh, held, B_held)

    while True:
        if s < 1.0:
            # advance the indenter and the gel together (module docstring)
            ds, w, B = choose(cand, lambda b: np.inf)
            if M + ds * B > margin:
                cand = BP.candidates(x, fr.y(s), pad, ind, r_inf)
                info.rebuilds += 1
                M = 0.0
                ds, w, B = choose(cand, lambda b: margin / b if b > 0 else np.inf)
            for _ in range(prm.max_halvings + 1):
                s1 = 1.0 if ds >= 1.0 - s else s + ds
                if np.isfinite(En.energy_only(fr, x + ds * w, s1, cand)):
                    break
                ds *= 0.5
            else:
                info.status = NONFINITE
                break
            x = x + ds * w
            s = s1
            M += ds * B
            info.substeps += 1
            info.min_gap = min(info.min_gap, min_distance(fr, x, s, cand))
        E, g, blk = En.total(fr, x, s, cand)
        if not np.isfinite(E):
            info.status = NONFINITE
            break
        P = precondition(blk, free, prm.precond)
        p = -apply_P(P, g)
        if g_ref is None:
            g_ref = max(pad.g_ref, float(np.abs(g[free]).max(initial=0.0)))
            info.g_ref = g_ref
        target = (prm.tol if s >= 1.0 else max(prm.tol, prm.tol_advance)) * g_ref
        retried = False
        while np.abs(g[free]).max(initial=0.0) > target and info.iters < prm.max_iter:
            pn = vnorm_max(p)
            gTp = float(np.sum(g * p))
            if pn == 0.0 or gTp >= 0.0:
                p = -apply_P(P, g)
                pn, gTp = vnorm_max(p), float(np.sum(g * p))
            literal = prm.step == "literal"
            a_up = dhat / (2.0 * pn)
            a_ccd = np.inf if literal else ccd_bound(fr, x, p, s, cand, prm.eta)
            jet = En.total_line(fr, x, p, s, cand)
            pHp = float(jet.dd)
            a_bar = -gTp / pHp if pHp > 0 else np.inf
            alpha = min(a_up, a_ccd, a_bar)
            if M + alpha * pn > margin:
                cand = BP.candidates(x, fr.y(s), pad, ind, r_inf)
                info.rebuilds += 1
                M = 0.0
                if not literal:
                    a_ccd = ccd_bound(fr, x, p, s, cand, prm.eta)
                alpha = min(a_up, a_ccd, a_bar)
            accepted = False
            for _ in range(prm.max_halvings + 1):
                R = remainder(fr, x, p, alpha, s, cand)
                # the literal rule (Eq. step_size) takes alpha as it is; only
                # a trial state outside the energy's domain (an inverted tet
                # or a closed gap, where E is +inf) is halved
                if (np.isfinite(R) if literal else R <= (1.0 - prm.armijo_c) * alpha * (-gTp)):
                    accepted = True
                    break
                alpha *= 0.5
                info.halvings += 1
            if not accepted:
                # one retry along the preconditioned steepest descent -P g
                # before the line search counts as failed
                if not retried and not literal:
                    retried = True
                    p = -apply_P(P, g)
                    continue
                info.status = LINESEARCH
                break
            retried = False
            x = x + alpha * p
            M += alpha * pn
            E_new, g_new, blk_new = En.total(fr, x, s, cand)
            if not np.isfinite(E_new):
                info.status = NONFINITE
                break
            if E_new > E + 1e-9 * abs(E):
                info.energy_monotone = False
            info.min_gap = min(info.min_gap, min_distance(fr, x, s, cand))
            P_new = precondition(blk_new, free, prm.precond)
            z = apply_P(P_new, g_new)
            beta = dk_beta(g_new, g_new - g, p, P_new)
            p = -z + beta * p
            if float(np.sum(g_new * p)) >= 0.0:
                p = -z
            g, P, E = g_new, P_new, E_new
            info.iters += 1
            if trace is not None:
                trace.append((alpha * pn, E, float(np.abs(g[free]).max())))
        if info.status != CONVERGED:
            break
        if s >= 1.0:
            if np.abs(g[free]).max(initial=0.0) > target:
                info.status = MAXITER
            break
        if info.substeps >= prm.max_substeps or info.iters >= prm.max_iter:
            info.status = MAXITER
            break
    info.grad_inf = float(np.abs(g[free]).max(initial=0.0)) if info.status != NONFINITE else np.inf
    new = State(x=x, v=(x - x_t) / h, pose=np.asarray(pose_next, np.float64).copy())
    return new, info


def markers(pad, x):
    """Marker displacement (u_x, u_y) = sum_i w_i (x_i - X_i), first two
    components, on the rest top-face triangle of each marker (Sec. 3.2)."""
    u = x - pad.rest
    return np.einsum("mk,mkc->mc", pad.marker_w, u[pad.marker_ids])[:, :2]


def run(pad, ind, poses, prm=Params()):
    """Run frames 1..F of a pose sequence [F+1, 6] from rest. Returns the
    list of states (frame 0 = rest) and infos."""
    st = rest_state(pad, poses[0])
    states, infos = [st], []
    for f in range(1, len(poses)):
        st, info = solve_frame(pad, ind, st, poses[f], prm)
        states.append(st)
        infos.append(info)
    return states, infos
