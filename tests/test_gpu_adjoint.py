"""GPU adjoint (tac_adjoint) against the FP64 oracle adjoint, which is itself
pinned to full-solve central differences (tests/test_oracle_adjoint.py),
and the torch.autograd.Function built on it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint as AD
from oracle import geometry as G
from oracle import newton as NW
from oracle import solver as SV
from paper_2603_28475_b300 import scenes as S

from _cases import MM, oracle_pad

pytestmark = pytest.mark.gpu

DH = 0.05 * MM


@pytest.fixture(scope="module")
def tac():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_28475_b300 import build
    build.build()
    from paper_2603_28475_b300 import tac as T
    return T


def _scene():
    pd = S.hex_pad((6 * MM, 6 * MM, 2 * MM), (4, 4, 2), marker_shape=(3, 3))
    mat = S.Material(mu_f=0.5)
    ind_s = S.icosphere(2 * MM, 1)
    z0 = 2 * MM + DH - S.lowest_z(ind_s.verts, np.zeros(3))
    p0 = np.array([0.0, 0.0, 0.0, 3 * MM, 3 * MM, z0])
    p1 = p0 + np.array([0, 0, 0, 0, 0, -0.08 * MM])
    p2 = p0 + np.array([0.02, -0.01, 0.0, 0.02 * MM, 0.0, -0.12 * MM])
    poses = np.stack([p0, p1, p2]).astype(np.float32)
    return pd, mat, ind_s, poses


def _oracle_solve(pad, ind, st_prev, pose):
    prm = SV.Params(tol=1e-6)
    st, info = SV.solve_frame(pad, ind, st_prev, pose, prm)
    assert info.status == SV.CONVERGED
    fr = AD.frame_of(pad, ind, st_prev, pose)
    x, _, _ = NW.newton_polish(fr, st.x, 1.0, prm, tol_rel=1e-13)
    return SV.State(x=x, v=(x - st_prev.x) / pad.h, pose=np.asarray(pose, np.float64))


@pytest.fixture(scope="module")
def oracle_ref():
    pd, mat, ind_s, poses = _scene()
    pad = oracle_pad(pd, mat)
    ind = G.build_indenter(ind_s.verts, ind_s.tris)
    P = poses.astype(np.float64)
    s0 = SV.rest_state(pad, P[0])
    s1 = _oracle_solve(pad, ind, s0, P[1])
    s2 = _oracle_solve(pad, ind, s1, P[2])
    c = np.random.default_rng(0).normal(size=(pd.markers.shape[0], 2))
    return pad, ind, s1, s2, c, AD.adjoint(pad, ind, s1, s2, c)


# The adjoint is taken at the frame's equilibrium, which the oracle reaches to
# 1e-13 (Newton); the GPU frames are solved down to a float32 floor of 32
# ulps of the largest corner force (the default 256 leaves the pose
# sensitivities, which follow the contact gaps closely, a few 1e-3 apart).
TIGHT = 1e-9
FLOOR = 32.0


def _gpu_batch(tac):
    pd, mat, ind_s, poses = _scene()
    w = S.Workload("adjoint", [pd], [mat], [ind_s], 1, poses[:, None, :])
    b = tac.batch_from_workload(w, tol=TIGHT, floor_ulps=FLOOR)
    b.reset(torch.tensor(poses[0]).reshape(1, 6))
    for f in (1, 2):
        b.set_indenter(torch.tensor(poses[f]).reshape(1, 6))
        st, _ = b.step()
        assert int(st.item()) == 0
    return b, w


def test_adjoint_matches_oracle(tac, oracle_ref):
    pad, ind, s1, s2, c, ref = oracle_ref
    b, w = _gpu_batch(tac)
    g, st, it = b.adjoint(torch.tensor(c, dtype=torch.float32))
    torch.cuda.synchronize()
    assert int(st.item()) == 0, int(st.item())
    got = g.cpu().numpy()[0]
    scale = np.abs(ref).max()
    for k in range(9):
        assert got[k] == pytest.approx(ref[k], rel=1e-3, abs=1e-4 * scale), (k, got, ref)
    b.close()


def test_adjoint_with_knn_markers_matches_oracle(tac, oracle_ref):
    """The adjoint's right-hand side through the kNN marker map (4 weighted
    nodes per marker, markers moved off the nodes)."""
    from _cases import f32
    pad0, ind, s1, s2, _, _ = oracle_ref
    pd, mat, ind_s, poses = _scene()
    pd.markers = (pd.markers + np.array([0.3 * MM, 0.2 * MM])).astype(np.float32)
    pad = G.build_pad(pd.rest, pd.tets, pd.fixed, pd.markers, f32(mat.E), f32(mat.nu), f32(mat.rho), f32(mat.h),
                      f32(mat.dhat), f32(mat.mu_f), marker_mode="knn")
    assert np.all(pad.marker_w[:, 3] > 0)
    c = np.random.default_rng(4).normal(size=(pd.markers.shape[0], 2))
    ref = AD.adjoint(pad, ind, s1, s2, c)
    w = S.Workload("adjoint_knn", [pd], [mat], [ind_s], 1, poses[:, None, :])
    b = tac.batch_from_workload(w, tol=TIGHT, marker=1, floor_ulps=FLOOR)
    b.reset(torch.tensor(poses[0]).reshape(1, 6))
    for f in (1, 2):
        b.set_indenter(torch.tensor(poses[f]).reshape(1, 6))
        st, _ = b.step()
        assert int(st.item()) == 0
    mk = b.markers().cpu().numpy().astype(np.float64)
    assert np.abs(mk - SV.markers(pad, s2.x)).max() <= 1e-4 * 2 * MM
    g, st, it = b.adjoint(torch.tensor(c, dtype=torch.float32))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    got = g.cpu().numpy()[0]
    scale = np.abs(ref).max()
    for k in range(9):
        assert got[k] == pytest.approx(ref[k], rel=1e-3, abs=1e-4 * scale), (k, got, ref)
    b.close()


def test_autograd_function_gives_the_adjoint(tac, oracle_ref):
    from paper_2603_28475_b300 import autograd as A
    pad, ind, s1, s2, c, ref = oracle_ref
    pd, mat, ind_s, poses = _scene()
    w = S.Workload("adjoint", [pd], [mat], [ind_s], 1, poses[:, None, :])
    b = tac.batch_from_workload(w, tol=TIGHT, floor_ulps=FLOOR)
    b.reset(torch.tensor(poses[0]).reshape(1, 6))
    b.set_indenter(torch.tensor(poses[1]).reshape(1, 6))
    b.step()
    ck = A.FrameCheckpoint(b, poses[1])
    base = b.get_params()
    lame = torch.tensor([[pad.lam, pad.mu]], dtype=torch.float64, requires_grad=True)
    mu_f = torch.tensor([pad.mu_f], dtype=torch.float64, requires_grad=True)
    pose = torch.tensor(poses[2].astype(np.float64).reshape(1, 6), requires_grad=True)
    m = A.frame_markers(b, ck, lame, mu_f, pose, base)
    loss = (torch.tensor(c, dtype=torch.float32, device=m.device) * m).sum()
    loss.backward()
    got = np.concatenate([lame.grad.numpy()[0], mu_f.grad.numpy(), pose.grad.numpy()[0]])
    scale = np.abs(ref).max()
    for k in range(9):
        assert got[k] == pytest.approx(ref[k], rel=2e-3, abs=2e-4 * scale), (k, got, ref)
    # the marker field of the forward pass is the frame's solution
    assert np.abs(m.detach().cpu().numpy() - SV.markers(pad, s2.x)).max() <= 1e-4 * 2 * MM
    b.close()


# --- sequences: tac_adjoint_frame and the differentiable step

def _p3(poses):
    return poses[2] + np.array([0.01, 0.0, -0.01, 0.03 * MM, 0.01 * MM, -0.03 * MM], np.float32)


@pytest.fixture(scope="module")
def oracle_seq():
    pd, mat, ind_s, poses = _scene()
    poses = np.concatenate([poses, _p3(poses)[None]]).astype(np.float32)
    pad = oracle_pad(pd, mat)
    ind = G.build_indenter(ind_s.verts, ind_s.tris)
    P = poses.astype(np.float64)
    states = [SV.rest_state(pad, P[0])]
    for f in (1, 2, 3):
        states.append(_oracle_solve(pad, ind, states[-1], P[f]))
    rng = np.random.default_rng(3)
    cs = [rng.normal(size=(pd.markers.shape[0], 2)) for _ in range(3)]
    gx = rng.normal(size=pad.rest.shape) * 1e-3
    gx[~pad.free] = 0.0
    return pad, ind, poses, states, cs, gx


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_frame_adjoint_matches_oracle(tac, oracle_seq):
    """Frame 3 with a downstream gradient on its end positions: all 15
    parameter sensitivities and the start-state gradients."""
    pad, ind, poses, states, cs, gx = oracle_seq
    th_o, dx_o, dv_o = AD.adjoint_frame(pad, ind, states[2], states[3], cs[2], gx)
    pd, mat, ind_s, _ = _scene()
    w = S.Workload("adjoint", [pd], [mat], [ind_s], 1, poses[:, None, :])
    b = tac.batch_from_workload(w, tol=TIGHT, floor_ulps=FLOOR)
    b.reset(torch.tensor(poses[0]).reshape(1, 6))
    for f in (1, 2, 3):
        b.set_indenter(torch.tensor(poses[f]).reshape(1, 6))
        st, _ = b.step()
        assert int(st.item()) == 0
    th, dx0, dv0, st, it = b.adjoint_frame(torch.tensor(cs[2], dtype=torch.float32),
                                           torch.tensor(gx, dtype=torch.float32))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    got = th.cpu().numpy()[0]
    scale = np.abs(th_o).max()
    for k in range(15):
        assert got[k] == pytest.approx(th_o[k], rel=1e-3, abs=1e-4 * scale), (k, got, th_o)
    assert _rel(dx0.cpu().numpy().astype(np.float64), dx_o) <= 1e-3
    assert _rel(dv0.cpu().numpy().astype(np.float64), dv_o) <= 1e-3
    # without a downstream gradient the first 9 entries are tac_adjoint's
    th2, _, _, _, _ = b.adjoint_frame(torch.tensor(cs[2], dtype=torch.float32))
    g9, _, _ = b.adjoint(torch.tensor(cs[2], dtype=torch.float32))
    assert np.allclose(th2.cpu().numpy()[0, :9], g9.cpu().numpy()[0], rtol=1e-6,
                       atol=1e-9 * np.abs(g9.cpu().numpy()).max())
    b.close()


def test_sequence_autograd_matches_oracle_sweep(tac, oracle_seq):
    """Three frames chained with TacStepFn; loss.backward() against the
    oracle's reverse sweep (Lame pair, friction, end poses of frames 1-3)."""
    from paper_2603_28475_b300 import autograd as A
    pad, ind, poses, states, cs, gx = oracle_seq
    ref = AD.adjoint_sequence(pad, ind, states, cs)
    pd, mat, ind_s, _ = _scene()
    w = S.Workload("adjoint", [pd], [mat], [ind_s], 1, poses[:, None, :])
    b = tac.batch_from_workload(w, tol=TIGHT, floor_ulps=FLOOR)
    b.reset(torch.tensor(poses[0]).reshape(1, 6))
    x0, v0 = b.get_state()
    lame = torch.tensor([[pad.lam, pad.mu]], dtype=torch.float64, requires_grad=True)
    mu_f = torch.tensor([pad.mu_f], dtype=torch.float64, requires_grad=True)
    P = torch.tensor(poses.astype(np.float64).reshape(4, 1, 6), requires_grad=True)
    m = A.sequence_markers(b, x0, v0, lame, mu_f, P)
    loss = sum((torch.tensor(c, dtype=torch.float32, device=m.device) * m[f]).sum() for f, c in enumerate(cs))
    loss.backward()
    got = np.concatenate([lame.grad.numpy()[0], mu_f.grad.numpy(), P.grad.numpy()[1:, 0].ravel()])
    scale = np.abs(ref).max()
    for k in range(ref.size):
        assert got[k] == pytest.approx(ref[k], rel=2e-3, abs=2e-4 * scale), (k, got, ref)
    b.close()


def test_relagged_frame_adjoint_matches_oracle(tac, oracle_seq):
    """lag_mode 1: frame 3's adjoint with its friction lag differentiated as
    a function of the frame's start state and start pose, against the
    oracle's relagged frame adjoint (which is pinned to full re-solves)."""
    pad, ind, poses, states, cs, gx = oracle_seq
    th_o, dx_o, dv_o = AD.adjoint_frame(pad, ind, states[2], states[3], cs[2], gx, relag=True)
    th_f, dx_f, _ = AD.adjoint_frame(pad, ind, states[2], states[3], cs[2], gx)
    assert _rel(dx_f, dx_o) > 1e-2                   # the lag term is not negligible here
    pd, mat, ind_s, _ = _scene()
    w = S.Workload("adjoint", [pd], [mat], [ind_s], 1, poses[:, None, :])
    b = tac.batch_from_workload(w, tol=TIGHT, floor_ulps=FLOOR)
    b.reset(torch.tensor(poses[0]).reshape(1, 6))
    for f in (1, 2, 3):
        b.set_indenter(torch.tensor(poses[f]).reshape(1, 6))
        st, _ = b.step()
        assert int(st.item()) == 0
    th, dx0, dv0, st, it = b.adjoint_frame(torch.tensor(cs[2], dtype=torch.float32),
                                           torch.tensor(gx, dtype=torch.float32), relag=True)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    got = th.cpu().numpy()[0]
    scale = np.abs(th_o).max()
    for k in range(15):
        assert got[k] == pytest.approx(th_o[k], rel=1e-3, abs=1e-4 * scale), (k, got, th_o)
    assert _rel(dx0.cpu().numpy().astype(np.float64), dx_o) <= 1e-3
    assert _rel(dv0.cpu().numpy().astype(np.float64), dv_o) <= 1e-3
    b.close()


def test_relagged_sequence_autograd_matches_oracle_sweep(tac, oracle_seq):
    """Three frames chained with TacStepFn(relag); loss.backward() against
    the oracle's relagged reverse sweep."""
    from paper_2603_28475_b300 import autograd as A
    pad, ind, poses, states, cs, gx = oracle_seq
    ref = AD.adjoint_sequence(pad, ind, states, cs, relag=True)
    pd, mat, ind_s, _ = _scene()
    w = S.Workload("adjoint", [pd], [mat], [ind_s], 1, poses[:, None, :])
    b = tac.batch_from_workload(w, tol=TIGHT, floor_ulps=FLOOR)
    b.reset(torch.tensor(poses[0]).reshape(1, 6))
    x0, v0 = b.get_state()
    lame = torch.tensor([[pad.lam, pad.mu]], dtype=torch.float64, requires_grad=True)
    mu_f = torch.tensor([pad.mu_f], dtype=torch.float64, requires_grad=True)
    P = torch.tensor(poses.astype(np.float64).reshape(4, 1, 6), requires_grad=True)
    m = A.sequence_markers(b, x0, v0, lame, mu_f, P, relag=True)
    loss = sum((torch.tensor(c, dtype=torch.float32, device=m.device) * m[f]).sum() for f, c in enumerate(cs))
    loss.backward()
    got = np.concatenate([lame.grad.numpy()[0], mu_f.grad.numpy(), P.grad.numpy()[1:, 0].ravel()])
    scale = np.abs(ref).max()
    for k in range(ref.size):
        assert got[k] == pytest.approx(ref[k], rel=2e-3, abs=2e-4 * scale), (k, got, ref)
    b.close()


def test_installed_frame_gives_the_same_adjoint(tac, oracle_seq):
    """tac_set_frame installs frame 3 from its start state, poses and end
    positions without solving; its adjoint equals the adjoint taken right
    after the frame's own solve (the end positions differ only by the
    float32 readback)."""
    pad, ind, poses, states, cs, gx = oracle_seq
    pd, mat, ind_s, _ = _scene()
    w = S.Workload("adjoint", [pd], [mat], [ind_s], 1, poses[:, None, :])
    b = tac.batch_from_workload(w, tol=TIGHT, floor_ulps=FLOOR)
    P = torch.tensor(poses).reshape(4, 1, 6)
    b.reset(P[0])
    for f in (1, 2):
        b.set_indenter(P[f])
        b.step()
    x0, v0 = b.get_state()
    b.reset(P[2])
    b.set_state(x0, v0)
    b.set_indenter(P[3])
    st, _ = b.step()
    assert int(st.item()) == 0
    x1, _ = b.get_state()
    c = torch.tensor(cs[2], dtype=torch.float32)
    g = torch.tensor(gx, dtype=torch.float32)
    thA, dxA, dvA, stA, _ = b.adjoint_frame(c, g)
    b.set_frame(x0, v0, P[2], x1, P[3])
    thB, dxB, dvB, stB, _ = b.adjoint_frame(c, g)
    assert int(stA.item()) == 0 and int(stB.item()) == 0
    a, bb = thA.cpu().numpy()[0], thB.cpu().numpy()[0]
    assert np.abs(a - bb).max() <= 1e-4 * np.abs(a).max(), (a, bb)
    assert _rel(dxB.cpu().numpy().astype(np.float64), dxA.cpu().numpy().astype(np.float64)) <= 1e-4
    assert _rel(dvB.cpu().numpy().astype(np.float64), dvA.cpu().numpy().astype(np.float64)) <= 1e-4
    b.close()
