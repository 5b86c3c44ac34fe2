"""Adjoint of one frame's equilibrium (oracle, FP64).

At the frame's minimiser x* the gradient g(x*; theta) vanishes on the free
DOFs, so for a loss L(markers(x*)) the implicit-function theorem gives

    dL/dtheta = -lambda^T dg/dtheta,      H lambda = dL/dx,

with H = dg/dx the exact Hessian at x* (oracle.newton.assemble). The
parameters are theta = (Lame lambda, Lame mu, friction mu_f, end pose of
the indenter: rotation vector (3), translation (3)); the barrier stiffness
kappa, the lag of the frame (x^t, y^t) and the solver tolerances are held
fixed. dg/dtheta:
  * Lame pair: g_elastic is linear in (mu, lambda) (the stress
    mu (F - F^-T) + lambda ln J F^-T), so dg/dlambda is the elastic gradient
    with (mu, lambda) = (0, 1) and dg/dmu the one with (1, 0);
  * mu_f: the lagged friction gradient is linear in mu_f;
  * pose: central difference (steps 1e-7 rad, 1e-10 m) of the total
    gradient in each pose component, the indenter vertices recomputed from
    the pose.

``adjoint_frame`` adds the sensitivities to the frame's start (positions,
velocities, start pose) with the frame's friction lag held fixed, and
``adjoint_sequence`` chains frames in a reverse sweep.
"""
from __future__ import annotations

import copy

import numpy as np

from . import broadphase as BP
from . import energy as En
from . import geometry as G
from . import newton as NW


def marker_transpose(pad, dL_dm):
    """dL/dx from dL/d(markers): the transpose of the marker readout, summed
    over every entry of a marker's map (3 barycentric or k kNN nodes)."""
    g = np.zeros_like(pad.rest)
    for m in range(pad.marker_ids.shape[0]):
        for k in range(pad.marker_ids.shape[1]):
            g[pad.marker_ids[m, k], :2] += pad.marker_w[m, k] * dL_dm[m]
    return g


def frame_of(pad, ind, state_prev, pose_next, prm_margin=1.0, lag=None):
    x_t = state_prev.x
    xhat = x_t + pad.h * state_prev.v
    y_t = G.indenter_world(ind.verts, state_prev.pose)
    y_n = G.indenter_world(ind.verts, pose_next)
    if lag is None:
        cand = BP.candidates(x_t, y_t, pad, ind, pad.dhat * (1.0 + prm_margin))
        lag = En.friction_lag(cand, x_t, y_t, pad, ind)
    return En.Frame(pad, ind, x_t, xhat, y_t, y_n, lag)


# central-difference steps in the pose: rotation vector (rad) and translation
# (m); a translation step must stay far below the contact gaps (~1e-6 m),
# where the barrier gradient is strongly nonlinear
FD_ROT, FD_TRANS = 1e-7, 1e-10


def _fd_step(m, fd_pose):
    return fd_pose if m < 3 else fd_pose * (FD_TRANS / FD_ROT)


def adjoint(pad, ind, state_prev, state_new, dL_dm, fd_pose=FD_ROT):
    """dL/dtheta [9] = (lambda, mu, mu_f, rotvec(3), translation(3)) for the
    frame from state_prev to state_new (state_new.x the converged x*)."""
    fr = frame_of(pad, ind, state_prev, state_new.pose)
    x = state_new.x
    r = 2.0 * pad.dhat
    pairs = BP.candidates(x, fr.y(1.0), pad, ind, r)
    H = NW.assemble(fr, x, 1.0, pairs)
    fdof = np.repeat(pad.free, 3)
    b = marker_transpose(pad, np.asarray(dL_dm, np.float64)).ravel()
    lam = np.zeros_like(b)
    lam[fdof] = np.linalg.solve(H[np.ix_(fdof, fdof)], b[fdof])
    lam = lam.reshape(-1, 3)

    def dot_free(g):
        return float(np.sum(lam[pad.free] * g[pad.free]))

    out = np.zeros(9)
    p_lam = copy.copy(pad)
    p_lam.mu, p_lam.lam = 0.0, 1.0
    _, g_l, _ = En.elastic(x, p_lam, blocks=False)
    p_mu = copy.copy(pad)
    p_mu.mu, p_mu.lam = 1.0, 0.0
    _, g_m, _ = En.elastic(x, p_mu, blocks=False)
    out[0] = -dot_free(g_l)
    out[1] = -dot_free(g_m)
    if pad.mu_f > 0 and fr.lag["lam"].size:
        p_f = copy.copy(pad)
        p_f.mu_f = 1.0
        _, g_f, _ = En.friction(fr.lag, x, fr.x_t, fr.y(1.0), fr.y_t, p_f)
        out[2] = -dot_free(g_f)
    pose = np.asarray(state_new.pose, np.float64)
    for m in range(6):
        gs = []
        hm = _fd_step(m, fd_pose)
        for sgn in (1.0, -1.0):
            q = pose.copy()
            q[m] += sgn * hm
            frq = En.Frame(pad, ind, fr.x_t, fr.xhat, fr.y_t, G.indenter_world(ind.verts, q), fr.lag)
            _, g, _ = En.total(frq, x, 1.0, pairs)
            gs.append(g)
        out[3 + m] = -dot_free((gs[0] - gs[1]) / (2.0 * hm))
    return out


def adjoint_frame(pad, ind, state_prev, state_new, dL_dm=None, dL_dx=None, lag=None, fd_pose=FD_ROT, fd_x=1e-10,
                  relag=False):
    """Adjoint of one frame of a sequence. The frame's friction lag (normal
    forces, contact normals, closest-point weights, from its start state) is
    a constant of the frame, as in the frame's solve; with ``relag`` the lag
    is instead a function of the start state and start pose, rebuilt from
    them (on the frame's start candidate set) in every difference below, so
    that dL/dx^t and the start-pose entries include the lag's dependence.

    The right-hand side is the loss gradient with respect to the frame's end
    positions: the marker readout's transpose of dL_dm [M, 2] plus dL_dx
    [V, 3] (what later frames contribute), either may be None. Returns
    (theta [15], dL/dx^t [V, 3], dL/dv^t [V, 3]) with theta = (Lame lambda,
    Lame mu, mu_f, end pose (6), start pose (6)), each -lambda^T dg/d(.):
      * the first 9 as in ``adjoint``;
      * start pose: central difference of g in the start pose (it enters the
        friction term through the indenter's displacement over the frame);
      * x^t: central difference of g in each free start coordinate, x-hat =
        x^t + h v^t moving with it (inertia and the friction displacement);
      * v^t: g is affine in x-hat with dg/dx-hat = -M, so dL/dv^t = h M lambda.
    """
    if relag and lag is not None:
        raise ValueError("relag rebuilds the lag from the start state; do not pass one")
    fr = frame_of(pad, ind, state_prev, state_new.pose, lag=lag)
    cand_t = BP.candidates(fr.x_t, fr.y_t, pad, ind, 2.0 * pad.dhat) if relag else None
    x = state_new.x
    pairs = BP.candidates(x, fr.y(1.0), pad, ind, 2.0 * pad.dhat)
    H = NW.assemble(fr, x, 1.0, pairs)
    fdof = np.repeat(pad.free, 3)
    b = np.zeros(x.size)
    if dL_dm is not None:
        b += marker_transpose(pad, np.asarray(dL_dm, np.float64)).ravel()
    if dL_dx is not None:
        b += np.asarray(dL_dx, np.float64).ravel()
    lam = np.zeros_like(b)
    lam[fdof] = np.linalg.solve(H[np.ix_(fdof, fdof)], b[fdof])
    lam = lam.reshape(-1, 3)

    def dot_free(g):
        return float(np.sum(lam[pad.free] * g[pad.free]))

    theta = np.zeros(15)
    p_lam = copy.copy(pad)
    p_lam.mu, p_lam.lam = 0.0, 1.0
    p_mu = copy.copy(pad)
    p_mu.mu, p_mu.lam = 1.0, 0.0
    theta[0] = -dot_free(En.elastic(x, p_lam, blocks=False)[1])
    theta[1] = -dot_free(En.elastic(x, p_mu, blocks=False)[1])
    if pad.mu_f > 0 and fr.lag["lam"].size:
        p_f = copy.copy(pad)
        p_f.mu_f = 1.0
        theta[2] = -dot_free(En.friction(fr.lag, x, fr.x_t, fr.y(1.0), fr.y_t, p_f)[1])

    def g_of(x_t=fr.x_t, xhat=fr.xhat, y_t=fr.y_t, y_n=fr.y_next):
        lg = En.friction_lag(cand_t, x_t, y_t, pad, ind) if relag else fr.lag
        return En.total(En.Frame(pad, ind, x_t, xhat, y_t, y_n, lg), x, 1.0, pairs)[1]

    pose_n = np.asarray(state_new.pose, np.float64)
    pose_t = np.asarray(state_prev.pose, np.float64)
    for m in range(6):
        hm = _fd_step(m, fd_pose)
        gs = []
        for sgn in (1.0, -1.0):
            q = pose_n.copy()
            q[m] += sgn * hm
            gs.append(g_of(y_n=G.indenter_world(ind.verts, q)))
        theta[3 + m] = -dot_free((gs[0] - gs[1]) / (2.0 * hm))
        gs = []
        for sgn in (1.0, -1.0):
            q = pose_t.copy()
            q[m] += sgn * hm
            gs.append(g_of(y_t=G.indenter_world(ind.verts, q)))
        theta[9 + m] = -dot_free((gs[0] - gs[1]) / (2.0 * hm))
    dx0 = np.zeros_like(x)
    for i in np.nonzero(pad.free)[0]:
        for c in range(3):
            gs = []
            for sgn in (1.0, -1.0):
                xt = fr.x_t.copy()
                xh = fr.xhat.copy()
                xt[i, c] += sgn * fd_x
                xh[i, c] += sgn * fd_x
                gs.append(g_of(x_t=xt, xhat=xh))
            dx0[i, c] = -dot_free((gs[0] - gs[1]) / (2.0 * fd_x))
    dv0 = pad.h * pad.mass[:, None] * lam
    dv0[~pad.free] = 0.0
    return theta, dx0, dv0


def adjoint_sequence(pad, ind, states, dL_dms, lags=None, relag=False):
    """dL/dtheta for L = sum_f dL_dms[f-1] . markers(x^f) over frames
    1..F of a run from states[0], each frame's friction lag held fixed
    (``lags[f-1]`` if given, else the lag of states[f-1]) or, with
    ``relag``, differentiated as a function of the frame's start state and
    start pose (the total derivative of a run whose frames each lag
    themselves). theta = (Lame
    lambda, Lame mu, mu_f, end pose of frame 1, ..., end pose of frame F)
    [3 + 6F]; frame 1's start pose is a constant.

    Reverse sweep: frame f's end state receives the markers' gradient plus
    a_x + a_v / h from frame f+1 (v^f = (x^f - x^(f-1)) / h); frame f then
    passes a_x = dL/dx^(f-1) - a_v / h and a_v = dL/dv^(f-1) on."""
    F = len(states) - 1
    out = np.zeros(3 + 6 * F)
    a_x = np.zeros_like(states[0].x)
    a_v = np.zeros_like(states[0].x)
    for f in range(F, 0, -1):
        th, dx0, dv0 = adjoint_frame(pad, ind, states[f - 1], states[f], dL_dms[f - 1], a_x + a_v / pad.h,
                                     lag=None if lags is None else lags[f - 1], relag=relag)
        out[0:3] += th[0:3]
        out[3 + 6 * (f - 1):3 + 6 * f] += th[3:9]
        if f >= 2:
            out[3 + 6 * (f - 2):3 + 6 * (f - 1)] += th[9:15]
        a_x = dx0 - a_v / pad.h
        a_v = dv0
    return out
