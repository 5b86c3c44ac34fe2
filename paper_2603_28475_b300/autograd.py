"""torch.autograd.Function over one frame of the batched solve.

forward(lame, mu_f, pose): restores the checkpointed pre-frame state, sets
the material and friction parameters and the indenter target pose, solves
the frame (tac_step) and returns the marker field. backward(dL/dmarkers)
calls tac_adjoint, the implicit-function adjoint of the frame's equilibrium,
for dL/d(lame, mu_f, pose). The barrier stiffness and the friction mollifier
width are held at the values the batch resolved when the function was
built; the pre-frame state (positions, velocities, start pose) is a
constant of the frame, so a sequence of frames is differentiated frame by
frame with each frame's own checkpoint.
"""
from __future__ import annotations

import copy

import torch

from . import tac as T


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
