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
  * pose: central difference (step 1e-7) of the total gradient in each pose
    component, the indenter vertices recomputed from the pose.
"""
from __future__ import annotations

import copy

import numpy as np

from . import broadphase as BP
from . import energy as En
from . import geometry as G
from . import newton as NW


def marker_transpose(pad, dL_dm):
    """dL/dx from dL/d(markers): the transpose of the barycentric readout."""
    g = np.zeros_like(pad.rest)
    for m in range(pad.marker_ids.shape[0]):
        for k in range(3):
            g[pad.marker_ids[m, k], :2] += pad.marker_w[m, k] * dL_dm[m]
    return g


def frame_of(pad, ind, state_prev, pose_next, prm_margin=1.0):
    x_t = state_prev.x
    xhat = x_t + pad.h * state_prev.v
    y_t = G.indenter_world(ind.verts, state_prev.pose)
    y_n = G.indenter_world(ind.verts, pose_next)
    cand = BP.candidates(x_t, y_t, pad, ind, pad.dhat * (1.0 + prm_margin))
    lag = En.friction_lag(cand, x_t, y_t, pad, ind)
    return En.Frame(pad, ind, x_t, xhat, y_t, y_n, lag)


def adjoint(pad, ind, state_prev, state_new, dL_dm, fd_pose=1e-7):
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
        for sgn in (1.0, -1.0):
            q = pose.copy()
            q[m] += sgn * fd_pose
            frq = En.Frame(pad, ind, fr.x_t, fr.xhat, fr.y_t, G.indenter_world(ind.verts, q), fr.lag)
            _, g, _ = En.total(frq, x, 1.0, pairs)
            gs.append(g)
        out[3 + m] = -dot_free((gs[0] - gs[1]) / (2.0 * fd_pose))
    return out
