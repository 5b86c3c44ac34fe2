"""The calibration drivers on the GPU (Sec. 4.2, Eq. loss_function; Supp. C).

Synthetic recordings are the marker fields at hidden parameters. Checked:
the batched loss of a population equals Eq. loss_function computed from a
separate single-candidate batch (pad layout, normalisation); the loss is 0
at the hidden parameters and positive away from them; CMA-ES (population
12) recovers the Poisson ratio and the friction coefficient from a
press-and-slide; the adjoint gradient of the same loss agrees with central
differences of the batched loss: in nu on a frictionless press-and-slide,
and in nu and mu_f with friction when the sweep differentiates each frame's
friction lag (relag). The frozen-lag sweep holds the lags fixed while the
differences re-solve and so re-lag every frame: with friction its mu_f
gradient still agrees, its nu gradient only in sign. The press is
displacement-controlled, so the quasi-static marker field depends on E only
through the fixed barrier stiffness and inertia: its loss sensitivity is
small and CMA-ES needs many more generations for it, so these tests
calibrate nu and mu_f (bench.py --calibrate runs all four parameters).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2603_28475_b300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_28475_b300 import build
    build.build()
    from paper_2603_28475_b300 import calibrate
    return calibrate


@pytest.fixture(scope="module")
def setup(C):
    w, _ = S.config_calibration(n_envs=2, frames=6, seed=1, pad_verts=2000)
    base = S.Material(E=1e5, nu=0.42, rho=1100.0, mu_f=1.4)
    cal = C.Calibration(w, 12, base, names=("nu", "mu_f"))
    truth = np.array([0.46, 0.8])
    tgt = cal.targets(truth)
    yield w, base, cal, truth, tgt
    cal.close()


def test_population_loss_is_eq_loss_function(C, setup):
    from paper_2603_28475_b300 import tac as T
    w, base, cal, truth, tgt = setup
    thetas = np.stack([truth + np.array([0.002, 0.02]) * k for k in range(12)])
    L = cal.loss(thetas, tgt)
    assert L[0] == 0.0 and np.all(L[1:] > 0)
    # candidate 5 alone, in a batch of its own
    m = S.Material(E=base.E, nu=float(thetas[5][0]), rho=base.rho, mu_f=float(thetas[5][1]))
    b = T.TacBatch(w.pads, [T.make_params(m, kappa=cal.kappa[i], eps_v=cal.eps_v[i]) for i in range(2)],
                   w.indenters, pads_per_env=1, pair_capacity=8192)
    poses = torch.tensor(w.poses, dtype=torch.float32, device=b.device)
    b.reset(poses[0])
    acc = 0.0
    for f in range(1, w.poses.shape[0]):
        b.set_indenter(poses[f])
        b.step()
        d = (b.markers() - tgt[f - 1]).double().cpu().numpy().reshape(2, -1)
        acc += float((d * d).sum(axis=1).sum())
    b.close()
    assert L[5] == pytest.approx(acc / (6 * 2), rel=1e-12)


def test_cmaes_recovers_poisson_ratio_and_friction(C, setup):
    w, base, cal, truth, tgt = setup
    best, hist = C.calibrate_cmaes(cal, tgt, generations=25, sigma0=0.25, seed=0)
    print("best", best, "truth", truth, "loss", hist.best_loss[0], "->", hist.best_loss[-1])
    assert abs(best[0] / truth[0] - 1) < 0.005
    assert abs(best[1] / truth[1] - 1) < 0.03
    assert hist.best_loss[-1] < 1e-3 * hist.best_loss[0]


def _adjoint_grad(C, w, base, cal, tgt, th0, relag=False):
    """Adjoint gradient of Eq. loss_function in (nu, mu_f) at th0 (E at base.E)."""
    from paper_2603_28475_b300 import autograd as A
    from paper_2603_28475_b300 import tac as T
    n = w.n_pads
    b = T.TacBatch(w.pads, [T.make_params(S.Material(E=base.E, nu=float(th0[0]), rho=base.rho, mu_f=float(th0[1])),
                                          kappa=cal.kappa[i], eps_v=cal.eps_v[i]) for i in range(n)],
                   w.indenters, pads_per_env=1, pair_capacity=8192)
    bp = b.get_params()
    poses = torch.tensor(w.poses.astype(np.float64), device=b.device)
    b.reset(poses[0].float())
    x0, v0 = b.get_state()
    nu = torch.tensor(th0[0], dtype=torch.float64, requires_grad=True)
    mf = torch.tensor(th0[1], dtype=torch.float64, requires_grad=True)
    E = base.E
    lame = torch.stack([E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))]).reshape(1, 2).expand(n, 2)
    m = A.sequence_markers(b, x0, v0, lame, mf.reshape(1).expand(n), poses, base_params=bp, relag=relag)
    F = w.poses.shape[0] - 1
    d = (m.double() - tgt.double()).reshape(F, n, -1)
    loss = (d * d).sum(dim=2).mean()
    loss.backward()
    b.close()
    return np.array([nu.grad.item(), mf.grad.item()])


def _fd(cal, tgt, th0, rel=1e-3):
    """Central differences of the batched loss in nu and, when th0's mu_f is
    positive, in mu_f (else nan)."""
    h = rel * np.abs(th0)
    th = np.repeat(th0[None], cal.P, 0)
    th[1, 0] += h[0]; th[2, 0] -= h[0]
    if h[1] > 0:
        th[3, 1] += h[1]; th[4, 1] -= h[1]
    L = cal.loss(th, tgt)
    return np.array([(L[1] - L[2]) / (2 * h[0]), (L[3] - L[4]) / (2 * h[1]) if h[1] > 0 else np.nan])


def test_adjoint_gradient_in_nu_matches_differences_without_friction(C, setup):
    w, _, _, _, _ = setup
    base = S.Material(E=1e5, nu=0.42, rho=1100.0, mu_f=0.0)
    cal = C.Calibration(w, 12, base, names=("nu", "mu_f"))
    tgt = cal.targets([0.46, 0.0])
    th0 = np.array([0.44, 0.0])
    fd = _fd(cal, tgt, th0)
    g = _adjoint_grad(C, w, base, cal, tgt, th0)
    cal.close()
    print("frictionless: adjoint", g, "fd", fd)
    assert g[0] == pytest.approx(fd[0], rel=0.02)


def test_adjoint_gradient_in_friction_matches_differences(C, setup):
    w, base, cal, truth, tgt = setup
    th0 = np.array([0.44, 0.6])
    fd = _fd(cal, tgt, th0)
    g = _adjoint_grad(C, w, base, cal, tgt, th0)
    gr = _adjoint_grad(C, w, base, cal, tgt, th0, relag=True)
    print("with friction: frozen-lag adjoint", g, "relagged", gr, "fd", fd)
    assert g[1] == pytest.approx(fd[1], rel=0.05)
    assert np.sign(g[0]) == np.sign(fd[0])
    # the relagged sweep is the total derivative of the re-solved loss
    assert np.allclose(gr, fd, rtol=0.02, atol=0)
