"""The calibration workload against targets the FP64 oracle wrote.

tests/golden/calibration_targets.npz holds, for the calibration workload's
first environments (5k pads, 16-frame press-and-slide, friction), the
marker fields the oracle solved at each environment's hidden (E, nu, mu_f)
with the nominal material's barrier stiffness and mollifier width (written
by tests/golden/make_calibration_targets.py, which calls only oracle/).
The GPU runs the same sixteen frames at the same materials from rest; its
marker fields must match the targets within 1e-4 of the gel thickness in
every frame. The misfit at the nominal material is then positive and its
adjoint gradient (the lag differentiated) points downhill: a step against
it lowers the loss.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_28475_b300 import scenes as S

from _cases import MM

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
TOL = 1e-4 * 4 * MM
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "calibration_targets.npz")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_28475_b300 import build
    build.build()
    from paper_2603_28475_b300 import tac as T
    g = np.load(GOLDEN)
    n = len(g["envs"])
    w_all, hidden = S.config_calibration(n_envs=256, frames=int(g["frames"]), seed=0)
    w = S.Workload("calibration_head", w_all.pads[:n], w_all.materials[:n], w_all.indenters[:n], 1,
                   w_all.poses[:, :n])
    return T, g, w, hidden[:n]


def _params(T, w, g, mats):
    out = []
    for k, m in enumerate(mats):
        out.append(T.make_params(m, kappa=float(g["kappa"][k]), eps_v=float(g["eps_v"][k])))
    return out


def test_gpu_reproduces_oracle_targets(setup):
    T, g, w, hidden = setup
    mats = [S.Material(E=h.E, nu=h.nu, rho=w.materials[k].rho, h=w.materials[k].h, dhat=w.materials[k].dhat,
                       mu_f=h.mu_f) for k, h in enumerate(hidden)]
    b = T.TacBatch(w.pads, _params(T, w, g, mats), w.indenters, pads_per_env=1)
    poses = torch.tensor(w.poses, dtype=torch.float32, device=b.device)
    b.reset(poses[0])
    worst = 0.0
    mo = b.marker_offsets
    for f in range(1, w.n_frames + 1):
        b.set_indenter(poses[f])
        st, it = b.step()
        assert (st == 0).all(), (f, st.cpu().numpy())
        mk = b.markers().cpu().numpy().astype(np.float64)
        for k in range(w.n_pads):
            err = np.abs(mk[mo[k]:mo[k + 1]] - g["markers"][k, f - 1]).max()
            worst = max(worst, err)
            assert err <= TOL, (f, k, err)
    b.close()
    print(f"{w.n_pads} envs x {w.n_frames} frames: max marker error vs oracle targets {worst:.2e} m "
          f"(tolerance {TOL:.1e} m)")


def test_adjoint_gradient_lowers_the_target_misfit(setup):
    from paper_2603_28475_b300 import autograd as A
    T, g, w, hidden = setup
    base = _params(T, w, g, w.materials)
    b = T.TacBatch(w.pads, base, w.indenters, pads_per_env=1)
    poses = torch.tensor(w.poses.astype(np.float64), device=b.device)
    targets = torch.tensor(g["markers"], dtype=torch.float32, device=b.device)     # [env, frame, m, 2]
    targets = targets.permute(1, 0, 2, 3).reshape(w.n_frames, -1, 2)
    b.reset(poses[0].float())
    x0, v0 = b.get_state()
    prm = b.get_params()
    lam = np.array([q.E * q.nu / ((1 + q.nu) * (1 - 2 * q.nu)) for q in prm])
    mu = np.array([q.E / (2 * (1 + q.nu)) for q in prm])

    def loss_at(lame_np, muf_np, grad=False):
        lame = torch.tensor(lame_np, dtype=torch.float64, requires_grad=grad)
        muf = torch.tensor(muf_np, dtype=torch.float64, requires_grad=grad)
        m = A.sequence_markers(b, x0, v0, lame, muf, poses, base_params=prm, relag=True)
        loss = ((m - targets) ** 2).sum()
        if grad:
            loss.backward()
            return float(loss.item()), lame.grad.numpy().copy(), muf.grad.numpy().copy()
        return float(loss.item())

    lame0 = np.stack([lam, mu], 1)
    muf0 = np.array([q.mu_f for q in prm])
    L0, gl, gm = loss_at(lame0, muf0, grad=True)
    assert L0 > 0 and np.all(np.isfinite(gl)) and np.all(np.isfinite(gm))
    # a small step against the gradient in the normalised coordinates lowers the loss
    scale = np.concatenate([lame0.ravel(), muf0])
    gvec = np.concatenate([gl.ravel(), gm]) * scale
    step = -1e-3 * gvec / np.abs(gvec).max()
    new = scale * (1.0 + step)
    L1 = loss_at(new[:lame0.size].reshape(lame0.shape), new[lame0.size:])
    b.close()
    print(f"misfit {L0:.4e} -> {L1:.4e} after a 1e-3 relative step against the adjoint gradient")
    assert L1 < L0


GRAD = os.path.join(os.path.dirname(__file__), "golden", "calibration_gradient.npz")


def test_sequence_adjoint_matches_oracle_central_differences(setup):
    """dL/d(E, nu, mu_f) of the first environment's 16-frame misfit against
    its oracle targets, at the nominal material: the GPU's relagged sequence
    adjoint (each frame's friction lag differentiated, the total derivative
    of the run) against the oracle's central differences in
    tests/golden/calibration_gradient.npz (written by
    tests/golden/make_calibration_gradient.py, which calls only oracle/),
    within 1e-3 relative. The forward frames solve to the same 1e-6 relative
    gradient with a 32-ulp float32 floor."""
    from paper_2603_28475_b300 import autograd as A
    T, g, w, hidden = setup
    gd = np.load(GRAD)
    w0 = S.Workload("calibration_env0", w.pads[:1], w.materials[:1], w.indenters[:1], 1, w.poses[:, :1])
    prm = [T.make_params(w0.materials[0], kappa=float(g["kappa"][0]), eps_v=float(g["eps_v"][0]), floor_ulps=32.0)]
    b = T.TacBatch(w0.pads, prm, w0.indenters, pads_per_env=1)
    poses = torch.tensor(w0.poses.astype(np.float64), device=b.device)
    target = torch.tensor(g["markers"][0], dtype=torch.float32, device=b.device)      # [frame, m, 2]
    b.reset(poses[0].float())
    x0, v0 = b.get_state()
    q = b.get_params()[0]
    E, nu = float(q.E), float(q.nu)
    assert np.allclose([E, nu, float(q.mu_f)], gd["theta0"], rtol=1e-7, atol=0)
    den = (1 + nu) * (1 - 2 * nu)
    lame = torch.tensor([[E * nu / den, E / (2 * (1 + nu))]], dtype=torch.float64, requires_grad=True)
    muf = torch.tensor([float(q.mu_f)], dtype=torch.float64, requires_grad=True)
    m = A.sequence_markers(b, x0, v0, lame, muf, poses, base_params=b.get_params(), adjoint_tol=1e-8, relag=True)
    loss = ((m.double() - target.double()) ** 2).sum()
    loss.backward()
    b.close()
    dl, dm = lame.grad.numpy()[0]
    # chain rule from (lambda, mu) to (E, nu)
    dE = dl * nu / den + dm / (2 * (1 + nu))
    dnu = dl * E * (1 + 2 * nu * nu) / den ** 2 - dm * E / (2 * (1 + nu) ** 2)
    got = np.array([dE, dnu, float(muf.grad.numpy()[0])])
    fd = gd["fd"][:, -1]
    rel = np.abs(got - fd) / np.abs(fd)
    print(f"misfit GPU {float(loss.item()):.6e} / oracle {float(gd['L0']):.6e}; dL/d(E, nu, mu_f) GPU {got} "
          f"oracle FD {fd}; relative errors {rel}")
    assert float(loss.item()) == pytest.approx(float(gd["L0"]), rel=5e-2)
    assert np.all(rel <= 1e-3), rel
