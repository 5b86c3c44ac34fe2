"""Pins of the oracle's PNCG iteration: Dai-Kou direction properties, the
Armijo remainder, solve invariants (monotone energy, no interpenetration),
Newton certification of the end point and marker readout."""
import numpy as np
import pytest

from oracle import broadphase as BP
from oracle import energy as En
from oracle import geometry as G
from oracle import newton as NW
from oracle import solver as SV

from _cases import MM, c1, small_indenter, tiny_pad


def _P(n, rng):
    A = rng.normal(size=(n, 3, 3))
    return A @ np.swapaxes(A, 1, 2) + 0.1 * np.eye(3)[None]


def test_dk_direction_sufficient_descent():
    """For any g, y, p and SPD P the direction -P g + beta p of Eq.
    (dk_direction) satisfies g^T p_new <= -3/4 g^T P g."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        n = 5
        P = _P(n, rng)
        g, y, p = rng.normal(size=(3, n, 3))
        beta = SV.dk_beta(g, y, p, P)
        pn = -SV.apply_P(P, g) + beta * p
        gPg = float(np.sum(g * SV.apply_P(P, g)))
        assert float(np.sum(g * pn)) <= -0.75 * gPg * (1 - 1e-12)


def test_dk_finite_termination_on_quadratic():
    """With exact line search on a strictly convex quadratic and a fixed
    preconditioner, DK reduces to preconditioned Hestenes-Stiefel CG, which
    terminates in at most n steps."""
    rng = np.random.default_rng(1)
    nv = 4
    n = 3 * nv
    A = rng.normal(size=(n, n))
    A = A @ A.T + n * np.eye(n)
    b = rng.normal(size=n)
    P = _P(nv, rng)

    def run(use_beta):
        x = np.zeros(n)
        g = (A @ x - b).reshape(nv, 3)
        p = -SV.apply_P(P, g)
        for _ in range(n):
            pf = p.ravel()
            alpha = -float(g.ravel() @ pf) / float(pf @ A @ pf)
            x = x + alpha * pf
            gn = (A @ x - b).reshape(nv, 3)
            beta = SV.dk_beta(gn, gn - g, p, P) if use_beta else 0.0
            p = -SV.apply_P(P, gn) + beta * p
            g = gn
        return np.abs(A @ x - b).max() / np.abs(b).max()
    assert run(True) < 1e-5            # n-step termination up to rounding
    assert run(False) > 1e-3           # steepest descent (beta = 0) is far from it


def test_remainder_is_second_order_and_consistent():
    w, pad, ind = c1()
    poses = w.poses[:, 0].astype(np.float64)
    st = SV.rest_state(pad, poses[0])
    st, _ = SV.solve_frame(pad, ind, st, poses[1])
    y = G.indenter_world(ind.verts, poses[1])
    pairs = BP.candidates(st.x, y, pad, ind, 2 * pad.dhat)
    fr = En.Frame(pad, ind, st.x, st.x + pad.h * st.v, y, y, En.friction_lag(pairs, st.x, y, pad, ind))
    rng = np.random.default_rng(2)
    p = rng.normal(size=st.x.shape) * pad.free[:, None] * 1e-3
    E0, g, _ = En.total(fr, st.x, 1.0, pairs)
    pHp = float(En.total_line(fr, st.x, p, 1.0, pairs).dd)
    for a in (1e-3, 1e-4):
        R = SV.remainder(fr, st.x, p, a, 1.0, pairs)
        assert R / a ** 2 == pytest.approx(0.5 * pHp, rel=2e-2)
    a = 2e-2
    E1 = En.energy_only(fr, st.x + a * p, 1.0, pairs)
    assert E1 - E0 == pytest.approx(a * float(np.sum(g * p)) + SV.remainder(fr, st.x, p, a, 1.0, pairs), rel=1e-6)


def test_no_motion_stays_at_rest():
    _, pad = tiny_pad()
    ind_s, ind = small_indenter()
    pose = np.array([0, 0, 0, 0, 0, 0.05])              # far above the pad
    st = SV.rest_state(pad, pose)
    new, info = SV.solve_frame(pad, ind, st, pose)
    assert info.status == SV.CONVERGED and info.iters == 0
    assert np.array_equal(new.x, pad.rest)


@pytest.fixture(scope="module")
def c1_run():
    w, pad, ind = c1()
    poses = w.poses[:, 0].astype(np.float64)[:4]
    states, infos = SV.run(pad, ind, poses)
    return w, pad, ind, poses, states, infos


def test_c1_frames_converge_monotonically_without_penetration(c1_run):
    w, pad, ind, poses, states, infos = c1_run
    for f, info in enumerate(infos):
        assert info.status == SV.CONVERGED
        assert info.energy_monotone
        assert info.grad_inf <= 1e-6 * info.g_ref and info.g_ref >= pad.g_ref
        assert 0 < info.min_gap
    # all-pairs check of the final state: every gel/indenter pair is separated
    y = G.indenter_world(ind.verts, poses[-1])
    ap = BP.all_pairs(pad, ind)
    d, _, _ = En.distances(ap, states[-1].x, y, pad, ind)
    assert d.min() > 0
    assert (d < pad.dhat).sum() > 0                      # the indenter is in contact


def test_c1_end_point_matches_newton(c1_run):
    w, pad, ind, poses, states, infos = c1_run
    xn, err, gi = NW.certify(pad, ind, states[2], states[3])
    thickness = 4 * MM
    assert gi <= 1e-10 * pad.g_ref
    assert err <= 1e-4 * thickness
    assert err <= 1e-5 * thickness                        # 10x inside the parity tolerance


def test_unloading_recovers_rest(c1_run):
    w, pad, ind, poses, states, infos = c1_run
    lift = poses[0].copy()
    lift[5] += 2 * MM
    st = states[-1]
    for _ in range(3):
        st, info = SV.solve_frame(pad, ind, st, lift)
        assert info.status == SV.CONVERGED
    disp = np.abs(states[-1].x - pad.rest).max()
    assert np.abs(st.x - pad.rest).max() < 2e-3 * disp


def test_markers_rest_and_rigid_translation():
    w, pad, ind = c1()
    assert np.abs(SV.markers(pad, pad.rest)).max() == 0.0
    t = np.array([1e-5, -2e-5, 3e-6])
    assert np.allclose(SV.markers(pad, pad.rest + t), t[:2], rtol=0, atol=1e-18)
    F = np.array([[1.01, 0.002, 0.0], [-0.003, 0.99, 0.0], [0.0, 0.0, 1.0]])
    x = pad.rest @ F.T
    mk = np.c_[pd_markers(w), np.zeros(len(pd_markers(w)))]
    ztop = pad.rest[:, 2].max()
    mk[:, 2] = ztop
    exact = (mk @ F.T - mk)[:, :2]
    assert np.allclose(SV.markers(pad, x), exact, rtol=0, atol=1e-12)


def pd_markers(w):
    return w.pads[0].markers.astype(np.float64)


def test_marker_weights_form_partition_of_unity():
    w, pad, ind = c1()
    assert np.allclose(pad.marker_w.sum(axis=1), 1.0)
    assert np.all(pad.marker_w >= -1e-12)
    Xq = np.einsum("mk,mkc->mc", pad.marker_w, pad.rest[pad.marker_ids])[:, :2]
    assert np.allclose(Xq, pd_markers(w), atol=1e-12)


def test_preconditioner_inverts_the_blocks_and_masks_dirichlet_vertices():
    """R6: block mode gives P_i = K_i^-1 (P_i K_i = I) on free vertices, the
    scalar mode the inverse of the blocks' diagonals; Dirichlet vertices get
    P = 0 in both, so z = P g never moves them."""
    rng = np.random.default_rng(5)
    n = 12
    A = rng.normal(size=(n, 3, 3))
    K = np.einsum("nij,nkj->nik", A, A) + 0.1 * np.eye(3)
    free = np.ones(n, bool)
    free[[0, 5, 11]] = False
    Pb = SV.precondition(K, free, "block")
    assert np.allclose(np.einsum("nij,njk->nik", Pb[free], K[free]), np.eye(3), atol=1e-10)
    assert np.all(Pb[~free] == 0.0)
    Ps = SV.precondition(K, free, "scalar")
    dg = np.einsum("nii->ni", K[free])
    assert np.allclose(Ps[free], np.einsum("ni,ij->nij", 1.0 / dg, np.eye(3)))
    assert np.all(Ps[~free] == 0.0)
    g = rng.normal(size=(n, 3))
    assert np.all(SV.apply_P(Pb, g)[~free] == 0.0)
    assert np.allclose(SV.apply_P(Pb, g)[free], np.linalg.solve(K[free], g[free][..., None])[..., 0])


def test_indenter_pose_is_rotation_vector_then_translation():
    """The pose (rotation vector, translation) of the indenter: a rotation by
    theta about z takes e_x to (cos theta, sin theta, 0); the rotation keeps
    every distance and orientation (det R = 1); the translation applies after
    it; a zero rotation vector is the identity."""
    Y = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 3.0], [1.0, 1.0, 1.0]])
    th = 0.3
    y = G.indenter_world(Y, [0.0, 0.0, th, 0.0, 0.0, 0.0])
    assert np.allclose(y[0], [np.cos(th), np.sin(th), 0.0], atol=1e-15)
    assert np.allclose(y[2], [0.0, 0.0, 3.0], atol=1e-15)
    rng = np.random.default_rng(2)
    rv, t = rng.normal(size=3) * 0.4, rng.normal(size=3) * 1e-3
    y = G.indenter_world(Y, np.concatenate([rv, t]))
    y0 = G.indenter_world(Y, np.concatenate([rv, np.zeros(3)]))
    assert np.allclose(y - y0, t, atol=1e-15)
    dY = np.linalg.norm(Y[:, None] - Y[None], axis=2)
    dy = np.linalg.norm(y0[:, None] - y0[None], axis=2)
    assert np.allclose(dY, dy, atol=1e-14)
    R = np.linalg.lstsq(Y[:3], y0[:3], rcond=None)[0].T
    assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(R @ rv, rv, atol=1e-12)                       # the axis stays fixed
    assert np.allclose(G.indenter_world(Y, np.zeros(6)), Y, atol=0)
