"""torch.autograd.Function over one frame of the batched solve.

forward(lame, mu_f, pose): restores the checkpointed pre-frame state, sets
the material and friction parameters and the indenter target pose, solves
the frame (tac_step) and returns the marker field. backward(dL/dmarkers)
calls tac_adjoint, the implicit-function adjoint of the frame's equilibrium,
for dL/d(lame, mu_f, pose). The barrier stiffness and the friction mollifier
width are held at the values the batch resolved when the function was
built; the pre-frame state (positions, velocities, start pose) is a
constant of the frame.

TacStepFn / sequence_markers differentiate a sequence: each frame is a
function of its start state as well, and its backward (tac_adjoint_frame)
returns the start state's gradient, so torch chains the frames into a
reverse sweep.
"""
from __future__ import annotations

import copy
import warnings

import torch

from . import tac as T


class NotConvergedWarning(UserWarning):
    """A frame's forward solve ended on a pad that did not converge, so its
    adjoint is taken at a state that is not an equilibrium."""


def _check_forward_status(status):
    """Warns when the forward solve of a frame left pads unconverged: the
    implicit-function adjoint assumes grad E = 0 at the end state."""
    bad = int((status != 0).sum().item())
    if bad:
        warnings.warn(f"{bad} pad(s) of the forward frame did not converge; the adjoint at their end state "
                      "is not the derivative of an equilibrium", NotConvergedWarning, stacklevel=3)


def lame_to_young(lam, mu):
    """(E, nu) of a Lame pair."""
    E = mu * (3.0 * lam + 2.0 * mu) / (lam + mu)
    nu = lam / (2.0 * (lam + mu))
    return E, nu


class FrameCheckpoint:
    """The state a frame starts from: positions, velocities, start pose."""

    def __init__(self, batch, start_pose):
        self.x, self.v = batch.get_state()
        self.pose = torch.as_tensor(start_pose, dtype=torch.float32, device=batch.device).reshape(batch.n_pads, 6)

    def restore(self, batch):
        batch.reset(self.pose)
        batch.set_state(self.x, self.v)


class TacFrameFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lame, mu_f, pose, batch, checkpoint, base_params, adjoint_tol=1e-6):
        checkpoint.restore(batch)
        prm = []
        lam_mu = lame.detach().double().cpu().numpy()
        muf = mu_f.detach().double().cpu().numpy()
        for k, base in enumerate(base_params):
            q = copy.copy(base)
            E, nu = lame_to_young(lam_mu[k, 0], lam_mu[k, 1])
            q.E, q.nu, q.mu_f = float(E), float(nu), float(muf[k])
            prm.append(q)
        batch.set_params(prm)
        batch.set_indenter(pose.detach().float().reshape(batch.n_pads, 6))
        status, iters = batch.step()
        ctx.batch = batch
        ctx.tol = adjoint_tol
        ctx.status = status
        ctx.like = (lame, mu_f, pose)
        return batch.markers().clone()

    @staticmethod
    def backward(ctx, grad_m):
        _check_forward_status(ctx.status)
        g, st, it = ctx.batch.adjoint(grad_m.contiguous(), tol=ctx.tol)
        lame, mu_f, pose = ctx.like
        to = lambda t, ref: t.to(device=ref.device, dtype=ref.dtype).reshape(ref.shape)
        return to(g[:, 0:2], lame), to(g[:, 2], mu_f), to(g[:, 3:9], pose), None, None, None, None


def frame_markers(batch, checkpoint, lame, mu_f, pose, base_params=None):
    """Marker field of one frame as a differentiable function of the Lame
    pair [n_pads, 2], friction [n_pads] and indenter end pose [n_pads, 6]."""
    if base_params is None:
        base_params = batch.get_params()
    return TacFrameFn.apply(lame, mu_f, pose, batch, checkpoint, base_params)


def _set_material(batch, base_params, lame, mu_f):
    prm = []
    lam_mu = lame.detach().double().cpu().numpy()
    muf = mu_f.detach().double().cpu().numpy()
    for k, base in enumerate(base_params):
        q = copy.copy(base)
        E, nu = lame_to_young(lam_mu[k, 0], lam_mu[k, 1])
        q.E, q.nu, q.mu_f = float(E), float(nu), float(muf[k])
        prm.append(q)
    batch.set_params(prm)


def _vertex_h(batch, base_params):
    """Per-vertex step size h [total_verts, 1] (caller vertex order)."""
    h = torch.empty(batch.total_verts, 1, dtype=torch.float32, device=batch.device)
    vo = batch.vert_offsets
    for k, base in enumerate(base_params):
        h[vo[k]:vo[k + 1]] = float(base.h)
    return h


class TacStepFn(torch.autograd.Function):
    """One frame as a differentiable function of its start state:
    (markers, x1, v1) = step(lame, mu_f, pose_start, pose_end, x0, v0).
    Chaining calls differentiates a sequence of frames: backward installs
    the frame from its saved start and end states (tac_set_frame, which
    rebuilds the frame's friction lag without solving; the batch holds one
    frame) and calls tac_adjoint_frame with the end state's gradient
    (markers, x1 and v1 = (x1 - x0) / h); the frame's friction lag is a
    constant of the frame."""

    @staticmethod
    def _solve(batch, base_params, lame, mu_f, pose_s, pose_e, x0, v0):
        _set_material(batch, base_params, lame, mu_f)
        batch.reset(pose_s.detach().float().reshape(batch.n_pads, 6))
        batch.set_state(x0.detach(), v0.detach())
        batch.set_indenter(pose_e.detach().float().reshape(batch.n_pads, 6))
        return batch.step()

    @staticmethod
    def forward(ctx, lame, mu_f, pose_s, pose_e, x0, v0, batch, base_params, adjoint_tol=1e-6, relag=False):
        status, _ = TacStepFn._solve(batch, base_params, lame, mu_f, pose_s, pose_e, x0, v0)
        x1, v1 = batch.get_state()
        m = batch.markers().clone()
        ctx.batch, ctx.base, ctx.tol, ctx.status, ctx.relag = batch, base_params, adjoint_tol, status, relag
        ctx.inputs = (lame.detach(), mu_f.detach(), pose_s.detach(), pose_e.detach(), x0.detach().clone(),
                      v0.detach().clone(), x1.clone())
        ctx.like = (lame, mu_f, pose_s, pose_e, x0, v0)
        return m, x1, v1

    @staticmethod
    def backward(ctx, gm, gx1, gv1):
        _check_forward_status(ctx.status)
        b = ctx.batch
        lame, mu_f, pose_s, pose_e, x0, v0, x1 = ctx.inputs
        _set_material(b, ctx.base, lame, mu_f)
        b.set_frame(x0, v0, pose_s.detach().float(), x1, pose_e.detach().float())
        hv = _vertex_h(b, ctx.base)
        zero = torch.zeros(b.total_verts, 3, dtype=torch.float32, device=b.device)
        gx1 = zero if gx1 is None else gx1.to(device=b.device, dtype=torch.float32)
        gv1 = zero if gv1 is None else gv1.to(device=b.device, dtype=torch.float32)
        th, dx0, dv0, st, it = b.adjoint_frame(gm, gx1 + gv1 / hv, tol=ctx.tol, relag=ctx.relag)
        gx0 = dx0 - gv1 / hv
        l_, m_, ps_, pe_, x_, v_ = ctx.like
        to = lambda t, ref: t.to(device=ref.device, dtype=ref.dtype).reshape(ref.shape)
        return (to(th[:, 0:2], l_), to(th[:, 2], m_), to(th[:, 9:15], ps_), to(th[:, 3:9], pe_), to(gx0, x_),
                to(dv0, v_), None, None, None, None)


def sequence_markers(batch, x0, v0, lame, mu_f, poses, base_params=None, adjoint_tol=1e-6, relag=False):
    """Marker fields of frames 1..F [F, total_markers, 2] from the start
    state (x0, v0) as a differentiable function of the Lame pair [n_pads, 2],
    friction [n_pads] and the poses [F + 1, n_pads, 6] (poses[0] the start
    pose of frame 1). relag: each frame's backward differentiates its
    friction lag as a function of the frame's start state and start pose
    (the total derivative of the run); otherwise the lag is a constant of
    its frame."""
    if base_params is None:
        base_params = batch.get_params()
    x, v, out = x0, v0, []
    for f in range(1, poses.shape[0]):
        m, x, v = TacStepFn.apply(lame, mu_f, poses[f - 1], poses[f], x, v, batch, base_params, adjoint_tol, relag)
        out.append(m)
    return torch.stack(out)
