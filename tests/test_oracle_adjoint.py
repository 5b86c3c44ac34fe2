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


def _solve(pad, ind, st_prev, pose):
    prm = SV.Params(tol=1e-6)           # Newton then polishes to 1e-13
    st, info = SV.solve_frame(pad, ind, st_prev, pose, prm)
    assert info.status == SV.CONVERGED
    fr = AD.frame_of(pad, ind, st_prev, pose)
    x, gi, _ = NW.newton_polish(fr, st.x, 1.0, prm, tol_rel=1e-13)
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
            vals.append(_loss(pk, _solve(pk, ind, s1, p2).x, c))
        fd[k] = (vals[0] - vals[1]) / (2 * h)
    for m in range(6):
        h = 1e-6 if m < 3 else 1e-6 * abs(p2[m])
        vals = []
        for sgn in (1.0, -1.0):
            q = p2.copy()
            q[m] += sgn * h
            vals.append(_loss(pad, _solve(pad, ind, s1, q).x, c))
        fd[3 + m] = (vals[0] - vals[1]) / (2 * h)
    scale = np.abs(fd).max()
    for k in range(9):
        assert got[k] == pytest.approx(fd[k], rel=1e-3, abs=1e-4 * scale), (k, got, fd)


def test_marker_transpose_is_the_adjoint_of_the_readout(setup):
    pad, ind, s1, s2, p2, c = setup
    rng = np.random.default_rng(1)
    u = rng.normal(size=pad.rest.shape)
    lhs = float(np.sum(c * SV.markers(pad, pad.rest + u)))
    rhs = float(np.sum(AD.marker_transpose(pad, c) * u))
    assert lhs == pytest.approx(rhs, rel=1e-12)
