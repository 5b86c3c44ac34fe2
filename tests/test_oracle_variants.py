"""Pins of the oracle's paper-literal variants.

* kNN inverse-distance markers (Sec. 3.2): exact brute force on a pad whose
  node coordinates are dyadic (every squared distance exact in FP64, ties
  exact), the defining property of inverse-distance weights (w_i d_i equal
  for all neighbours), the symmetric cell-centre case (four corners at 1/4),
  a marker on a node (weight 1), and reproduction of constant fields;
* the literal step rule of Eq. (step_size) and the scalar Jacobi
  preconditioner: each frame converges and its end point is the frame's
  minimiser, certified by the Newton check independently of the step rule.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import geometry as G
from oracle import newton as NW
from oracle import solver as SV
from paper_2603_28475_b300 import scenes as S

from _cases import MM, c1

SP = 2.0 ** -9            # grid spacing, exact in binary
CELLS = (6, 4, 2)


def _dyadic_pad():
    pd = S.hex_pad((CELLS[0] * SP, CELLS[1] * SP, CELLS[2] * SP), CELLS, marker_shape=(3, 3))
    assert np.all(pd.rest / SP == np.round(pd.rest / SP))      # nodes exactly on the lattice
    return pd


def _exact_knn(rest, q, k):
    """The k nearest top-face nodes by exact rational squared distance, ties
    to the smaller id (the reading's order), by sorting all candidates."""
    ztop = max(Fraction(float(z)) for z in rest[:, 2])
    qx, qy = Fraction(float(q[0])), Fraction(float(q[1]))
    keyed = []
    for i, X in enumerate(rest):
        if Fraction(float(X[2])) != ztop:
            continue
        dx, dy = Fraction(float(X[0])) - qx, Fraction(float(X[1])) - qy
        keyed.append((dx * dx + dy * dy, i))
    keyed.sort()
    return [i for _, i in keyed[:k]], [d for d, _ in keyed[:k]]


def test_knn_neighbours_match_exact_brute_force():
    pd = _dyadic_pad()
    rng = np.random.default_rng(3)
    # markers on a 1/8-cell lattice (dyadic), many of them at exact ties
    mk = rng.integers(0, 8 * np.array(CELLS[:2]) + 1, size=(60, 2)) * (SP / 8)
    ids, w = G.marker_map_knn(pd.rest, mk)
    for m, q in enumerate(mk):
        ref, d2 = _exact_knn(pd.rest, q, 4)
        assert ids[m].tolist() == ref, (m, q / SP)
        if d2[0] == 0:
            assert w[m].tolist() == [1.0, 0.0, 0.0, 0.0]
        else:
            d = np.sqrt([float(v) for v in d2])
            wd = w[m] * d
            assert np.allclose(wd, wd[0], rtol=1e-14, atol=0)     # w_i proportional to 1/d_i
            assert w[m].sum() == pytest.approx(1.0, abs=1e-15)


def test_knn_symmetric_and_degenerate_cases():
    pd = _dyadic_pad()
    X = pd.rest
    top = np.flatnonzero(X[:, 2] == X[:, 2].max())
    # cell centre: the four corners of the cell, equal weights
    q = np.array([[2.5 * SP, 1.5 * SP]])
    ids, w = G.marker_map_knn(X, q)
    corners = {int(i) for i in top if abs(X[i, 0] / SP - 2.5) == 0.5 and abs(X[i, 1] / SP - 1.5) == 0.5}
    assert set(ids[0].tolist()) == corners and len(corners) == 4
    assert np.array_equal(w[0], np.full(4, 0.25))
    # a marker on a node takes that node alone
    j = int(top[7])
    ids, w = G.marker_map_knn(X, X[j:j + 1, :2])
    assert ids[0, 0] == j and w[0].tolist() == [1.0, 0.0, 0.0, 0.0]


def test_knn_markers_reproduce_constant_fields():
    pd = _dyadic_pad()
    pad = G.build_pad(pd.rest, pd.tets, pd.fixed, pd.markers, 0.3e6, 0.45, 1100.0, 1 / 60, 0.05 * MM, 0.0,
                      marker_mode="knn")
    assert pad.marker_ids.shape == (len(pd.markers), 4)
    assert np.abs(SV.markers(pad, pad.rest)).max() == 0.0
    t = np.array([1.5e-4, -2.5e-4, 3e-5])
    assert np.allclose(SV.markers(pad, pad.rest + t), t[:2], rtol=0, atol=1e-18)
    assert np.all(pad.marker_w >= 0) and np.allclose(pad.marker_w.sum(axis=1), 1.0, rtol=0, atol=1e-15)


@pytest.fixture(scope="module")
def c1_frame():
    w, pad, ind = c1()
    poses = w.poses[:, 0].astype(np.float64)[:4]
    states, _ = SV.run(pad, ind, poses[:3])
    return pad, ind, poses, states[-1]


@pytest.mark.parametrize("prm", [SV.Params(step="literal"), SV.Params(precond="scalar")],
                         ids=["literal_step", "scalar_jacobi"])
def test_variant_reaches_the_newton_minimiser(c1_frame, prm):
    pad, ind, poses, st = c1_frame
    new, info = SV.solve_frame(pad, ind, st, poses[3], prm)
    assert info.status == SV.CONVERGED
    assert info.grad_inf <= 1e-6 * info.g_ref
    assert info.min_gap > 0
    _, err, gi = NW.certify(pad, ind, st, new)
    assert gi <= 1e-9 * pad.g_ref            # the polish's rounding floor
    assert err <= 1e-5 * 4 * MM
