"""Pin of the oracle's frame adjoint against FP64 central finite differences
of fully re-solved frames (Newton-polished), on a small pad with the friction
lag active."""
import copy

import numpy as np
import pytest

from oracle import adjoint as AD
from oracle import geometry as G
from oracle import newton as NW
from oracle import solver as SV
from paper_2603_28475_b300 import scenes as S

from _cases import MM

DH = 0.05 * MM


def _scene():
    pd = S.hex_pad((6 * MM, 6 * MM, 2 * MM), (4, 4, 2), marker_shape=(3, 3))
    pad = G.build_pad(pd.rest, pd.tets, pd.fixed, pd.markers, 0.3e6, 0.45, 1100.0, 1 / 60, DH, 0.5)
    ind_s = S.icosphere(2 * MM, 1)
    ind = G.build_indenter(ind_s.verts, ind_s.tris)
    z0 = 2 * MM + DH - S.lowest_z(ind_s.verts, np.zeros(3))
    p0 = np.array([0.0, 0.0, 0.0, 3 * MM, 3 * MM, z0])
    p1 = p0 + np.array([0, 0, 0, 0, 0, -0.08 * MM])
    p2 = p0 + np.array([0.02, -0.01, 0.0, 0.02 * MM, 0.0, -0.12 * MM])
    return pad, ind, p0, p1, p2


def _solve(pad, ind, st_prev, pose, x_init=None):
    """Frame equilibrium to 1e-13: PNCG then Newton, or, for a re-solve under
    a 1e-6 perturbation, Newton (exact Hessian) from the base equilibrium
    x_init, which lies in the basin of the nearby minimiser."""
    prm = SV.Params(tol=1e-6)
    fr = AD.frame_of(pad, ind, st_prev, pose)
    if x_init is None:
        st, info = SV.solve_frame(pad, ind, st_prev, pose, prm)
        assert info.status == SV.CONVERGED
        x_init = st.x
    x, gi, _ = NW.newton_polish(fr, x_init, 1.0, prm, tol_rel=1e-13)
    return SV.State(x=x, v=(x - st_prev.x) / pad.h, pose=np.asarray(pose, np.float64))


@pytest.fixture(scope="module")
def setup():
    pad, ind, p0, p1, p2 = _scene()
    s0 = SV.rest_state(pad, p0)
    s1 = _solve(pad, ind, s0, p1)
    s2 = _solve(pad, ind, s1, p2)
    fr = AD.frame_of(pad, ind, s1, p2)
    assert fr.lag["lam"].size > 0                     # friction is active in frame 2
    rng = np.random.default_rng(0)
    c = rng.normal(size=(pad.marker_ids.shape[0], 2))
    return pad, ind, s1, s2, p2, c


def _loss(pad, x, c):
    return float(np.sum(c * SV.markers(pad, x)))


def test_adjoint_matches_central_differences(setup):
    pad, ind, s1, s2, p2, c = setup
    got = AD.adjoint(pad, ind, s1, s2, c)
    fd = np.zeros(9)
    # Lame lambda, Lame mu, friction (kappa and the lag held fixed)
    for k, (attr, rel) in enumerate((("lam", 1e-6), ("mu", 1e-6), ("mu_f", 1e-6))):
        v0 = getattr(pad, attr)
        h = rel * v0
        vals = []
        for sgn in (1.0, -1.0):
            pk = copy.copy(pad)
            setattr(pk, attr, v0 + sgn * h)
            vals.append(_loss(pk, _solve(pk, ind, s1, p2, x_init=s2.x).x, c))
        fd[k] = (vals[0] - vals[1]) / (2 * h)
    for m in range(6):
        h = 1e-6 if m < 3 else 1e-6 * abs(p2[m])
        vals = []
        for sgn in (1.0, -1.0):
            q = p2.copy()
            q[m] += sgn * h
            vals.append(_loss(pad, _solve(pad, ind, s1, q, x_init=s2.x).x, c))
        fd[3 + m] = (vals[0] - vals[1]) / (2 * h)
    scale = np.abs(fd).max()
    for k in range(9):
        assert got[k] == pytest.approx(fd[k], rel=1e-3, abs=1e-4 * scale), (k, got, fd)


@pytest.mark.parametrize("mode", ["bary", "knn"])
def test_marker_transpose_is_the_adjoint_of_the_readout(setup, mode):
    pad, ind, s1, s2, p2, c = setup
    if mode == "knn":
        pd = S.hex_pad((6 * MM, 6 * MM, 2 * MM), (4, 4, 2), marker_shape=(3, 3))
        mk = pd.markers + np.array([0.3 * MM, 0.2 * MM])      # off the nodes: four weighted neighbours
        pad = G.build_pad(pd.rest, pd.tets, pd.fixed, mk, 0.3e6, 0.45, 1100.0, 1 / 60, DH, 0.5,
                          marker_mode="knn")
        assert pad.marker_ids.shape[1] == 4 and np.all(pad.marker_w[:, 3] > 0)
    rng = np.random.default_rng(1)
    u = rng.normal(size=pad.rest.shape)
    lhs = float(np.sum(c * SV.markers(pad, pad.rest + u)))
    rhs = float(np.sum(AD.marker_transpose(pad, c) * u))
    assert lhs == pytest.approx(rhs, rel=1e-12)


# --- sequence adjoint (reverse sweep over frames, each frame's lag held fixed)

def _solve_lag(pad, ind, st_prev, pose, lag):
    prm = SV.Params(tol=1e-6)
    st, info = SV.solve_frame(pad, ind, st_prev, pose, prm, lag=lag)
    assert info.status == SV.CONVERGED
    fr = AD.frame_of(pad, ind, st_prev, pose, lag=lag)
    x, _, _ = NW.newton_polish(fr, st.x, 1.0, prm, tol_rel=1e-13)
    return SV.State(x=x, v=(x - st_prev.x) / pad.h, pose=np.asarray(pose, np.float64))


def _run_seq(pad, ind, poses, lags):
    """Frames 1..F from rest; lags[f-1] is frame f's lag (None: its own)."""
    states, used = [SV.rest_state(pad, poses[0])], []
    for f in range(1, len(poses)):
        lag = lags[f - 1] if lags is not None else AD.frame_of(pad, ind, states[-1], poses[f]).lag
        used.append(lag)
        states.append(_solve_lag(pad, ind, states[-1], poses[f], lag))
    return states, used


@pytest.fixture(scope="module")
def seq_setup():
    pad, ind, p0, p1, p2 = _scene()
    p3 = p2 + np.array([0.01, 0.0, -0.01, 0.03 * MM, 0.01 * MM, -0.03 * MM])
    poses = np.stack([p0, p1, p2, p3])
    states, lags = _run_seq(pad, ind, poses, None)
    assert lags[2]["lam"].size > 0                    # friction active in the last frames
    rng = np.random.default_rng(2)
    cs = [rng.normal(size=(pad.marker_ids.shape[0], 2)) for _ in range(3)]
    return pad, ind, poses, states, lags, cs


def _seq_loss(pad, states, cs):
    return float(sum(np.sum(c * SV.markers(pad, s.x)) for c, s in zip(cs, states[1:])))


def test_sequence_adjoint_matches_central_differences(seq_setup):
    """Friction and frame 1's end-pose x (tangential, through friction) and z
    (normal) translations, each of which also sets frame 2's start pose and,
    through frame 1's end state, frames 2 and 3, against central differences
    of the 3-frame loss re-solved with the base lags. The Lame pair enters
    the chain exactly as mu_f does."""
    pad, ind, poses, states, lags, cs = seq_setup
    got = AD.adjoint_sequence(pad, ind, states, cs, lags=lags)
    checks = [("mu_f", 2), ("pose", 3 + 3), ("pose", 3 + 5)]
    fd = {}
    for attr, k in checks:
        vals = []
        if attr == "pose":
            f, m = divmod(k - 3, 6)
            h = 1e-6 if m < 3 else 1e-6 * abs(poses[f + 1][m])
            for sgn in (1.0, -1.0):
                q = poses.copy()
                q[f + 1, m] += sgn * h
                vals.append(_seq_loss(pad, _run_seq(pad, ind, q, lags)[0], cs))
        else:
            v0 = getattr(pad, attr)
            h = 1e-6 * v0
            for sgn in (1.0, -1.0):
                pk = copy.copy(pad)
                setattr(pk, attr, v0 + sgn * h)
                vals.append(_seq_loss(pk, _run_seq(pk, ind, poses, lags)[0], cs))
        fd[k] = (vals[0] - vals[1]) / (2 * h)
    scale = max(abs(v) for v in fd.values())
    for k, v in fd.items():
        assert got[k] == pytest.approx(v, rel=1e-3, abs=1e-4 * scale), (k, got[k], v)


def test_relagged_sequence_adjoint_matches_full_re_solves(seq_setup):
    """With the lag differentiated (relag), the sweep is the total
    derivative of a run whose frames each lag themselves: central
    differences of the 3-frame loss with every frame re-solved from its own
    start state and its own lag, for friction and frame 1's end-pose x and
    z translations (which reach frames 2 and 3 through their start states
    and start poses, and so through their lags)."""
    pad, ind, poses, states, lags, cs = seq_setup
    got = AD.adjoint_sequence(pad, ind, states, cs, relag=True)
    checks = [("mu_f", 2), ("pose", 3 + 3), ("pose", 3 + 5)]
    fd = {}
    for attr, k in checks:
        vals = []
        if attr == "pose":
            f, m = divmod(k - 3, 6)
            h = 1e-6 if m < 3 else 1e-6 * abs(poses[f + 1][m])
            for sgn in (1.0, -1.0):
                q = poses.copy()
                q[f + 1, m] += sgn * h
                vals.append(_seq_loss(pad, _run_seq(pad, ind, q, None)[0], cs))
        else:
            v0 = getattr(pad, attr)
            h = 1e-6 * v0
            for sgn in (1.0, -1.0):
                pk = copy.copy(pad)
                setattr(pk, attr, v0 + sgn * h)
                vals.append(_seq_loss(pk, _run_seq(pk, ind, poses, None)[0], cs))
        fd[k] = (vals[0] - vals[1]) / (2 * h)
    scale = max(abs(v) for v in fd.values())
    for k, v in fd.items():
        assert got[k] == pytest.approx(v, rel=1e-3, abs=1e-4 * scale), (k, got[k], v)


def test_frame_adjoint_reduces_to_single_frame_form(seq_setup):
    """With no downstream gradient, the first 9 entries are the single-frame
    adjoint and dL/dv^t = h M lambda vanishes on Dirichlet vertices."""
    pad, ind, poses, states, lags, cs = seq_setup
    th, dx0, dv0 = AD.adjoint_frame(pad, ind, states[1], states[2], cs[1])
    ref = AD.adjoint(pad, ind, states[1], states[2], cs[1])
    assert np.allclose(th[:9], ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    assert np.all(dv0[~pad.free] == 0.0) and np.all(dx0[~pad.free] == 0.0)
