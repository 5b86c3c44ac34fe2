"""Pins of the oracle's distances, barrier, friction and candidate set:
brute-force sampling, special cases, finite differences, C^k checks and an
all-pairs search."""
import numpy as np
import pytest

from oracle import broadphase as BP
from oracle import energy as En
from oracle import geometry as G
from oracle import newton as NW
from oracle import taylor as T

from _cases import MM, small_indenter, tiny_pad

DH = 0.05 * MM


# ---------------------------------------------------------------------------
# distances


def _sample_tri(A, B, C, n=160):
    u, v = np.meshgrid(np.linspace(0, 1, n + 1), np.linspace(0, 1, n + 1))
    m = u + v <= 1
    u, v = u[m], v[m]
    return A[None] + u[:, None] * (B - A)[None] + v[:, None] * (C - A)[None]


def _sample_seg(A, B, n=2000):
    t = np.linspace(0, 1, n + 1)
    return A[None] + t[:, None] * (B - A)[None]


def test_point_triangle_against_dense_sampling():
    rng = np.random.default_rng(0)
    for _ in range(40):
        A, B, C = rng.normal(size=(3, 3))
        P = rng.normal(size=3) * 1.5
        d, bary = En.point_triangle(P[None], A[None], B[None], C[None])
        S = _sample_tri(A, B, C)
        dmin = np.linalg.norm(S - P, axis=1).min()
        h = max(np.linalg.norm(B - A), np.linalg.norm(C - A), np.linalg.norm(C - B)) / 160
        assert d[0] <= dmin + 1e-12
        assert d[0] >= dmin - h
        Q = bary[0, 0] * A + bary[0, 1] * B + bary[0, 2] * C
        assert np.linalg.norm(P - Q) == pytest.approx(d[0], rel=1e-12)
        assert np.all(bary >= -1e-12) and bary.sum() == pytest.approx(1.0)


def test_point_over_face_is_plane_distance():
    A, B, C = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    P = np.array([0.25, 0.25, 0.3])
    d, bary = En.point_triangle(P[None], A[None], B[None], C[None])
    assert d[0] == pytest.approx(0.3)
    assert np.allclose(bary[0], [0.5, 0.25, 0.25])


def test_segment_segment_against_dense_sampling():
    rng = np.random.default_rng(1)
    for _ in range(40):
        P0, P1, Q0, Q1 = rng.normal(size=(4, 3))
        d, s, t = En.segment_segment(P0[None], P1[None], Q0[None], Q1[None])
        SP, SQ = _sample_seg(P0, P1, 400), _sample_seg(Q0, Q1, 400)
        D = np.linalg.norm(SP[:, None] - SQ[None], axis=2).min()
        h = (np.linalg.norm(P1 - P0) + np.linalg.norm(Q1 - Q0)) / 400
        assert d[0] <= D + 1e-12
        assert d[0] >= D - h
        r = (P0 + s[0] * (P1 - P0)) - (Q0 + t[0] * (Q1 - Q0))
        assert np.linalg.norm(r) == pytest.approx(d[0], rel=1e-12)


def test_parallel_segments():
    P0, P1 = np.array([0.0, 0, 0]), np.array([1.0, 0, 0])
    Q0, Q1 = np.array([0.5, 0.2, 0]), np.array([2.0, 0.2, 0])
    d, _, _ = En.segment_segment(P0[None], P1[None], Q0[None], Q1[None])
    assert d[0] == pytest.approx(0.2)


def _pair_setup(seed=0):
    """Tiny pad with a small icosphere placed within dhat of the top face so
    that candidates of all three types exist."""
    pd, pad = tiny_pad(cells=(3, 3, 1), size=(3 * MM, 3 * MM, 1 * MM), jitter=0.1, seed=seed)
    ind_s, ind = small_indenter(radius=0.6 * MM, subdiv=1)
    ztop = pad.rest[:, 2].max()
    pose = np.array([0.3, -0.2, 0.1, 1.4 * MM, 1.6 * MM, 0.0])
    y0 = G.indenter_world(ind.verts, pose)
    pose[5] = ztop - y0[:, 2].min() + 0.3 * DH
    y = G.indenter_world(ind.verts, pose)
    return pad, ind, y


def test_distance_gradient_is_weighted_normal():
    pad, ind, y = _pair_setup()
    pairs = BP.candidates(pad.rest, y, pad, ind, 2 * DH)
    assert set(np.unique(pairs[:, 0])) == {0, 1, 2}
    x = pad.rest
    d, w, (ty, gid, iid) = En.distances(pairs, x, y, pad, ind)
    P = En._slot_positions(gid, iid, x, y)
    r = np.einsum("ns,nsk->nk", w, P)
    rhat = r / d[:, None]
    h = 1e-10
    for k in range(0, len(pairs), max(1, len(pairs) // 40)):
        for sl in range(4):
            v = gid[k, sl]
            if v < 0:
                continue
            for c in range(3):
                xp, xm = x.copy(), x.copy()
                xp[v, c] += h
                xm[v, c] -= h
                dp, _, _ = En.distances(pairs[k:k + 1], xp, y, pad, ind)
                dm, _, _ = En.distances(pairs[k:k + 1], xm, y, pad, ind)
                # a vertex may appear in several slots of one pair only for edges sharing it: not here
                assert (dp[0] - dm[0]) / (2 * h) == pytest.approx(w[k, sl] * rhat[k, c], abs=1e-5)


# ---------------------------------------------------------------------------
# barrier


def test_barrier_closed_form_derivatives():
    d = np.linspace(0.02, 0.99, 50) * DH
    j = En.barrier(T.Jet(d, np.ones_like(d)), DH)
    assert np.allclose(j.d, En.barrier_d1(d, DH), rtol=1e-10)
    assert np.allclose(j.dd, En.barrier_d2(d, DH), rtol=1e-10)
    assert np.all(En.barrier(d, DH) > 0) and np.all(En.barrier_d1(d, DH) < 0) and np.all(En.barrier_d2(d, DH) > 0)


def test_barrier_is_c2_at_dhat():
    e = DH * np.array([1e-3, 1e-4, 1e-5])
    below = DH - e
    assert np.all(np.abs(En.barrier(below, DH)) < 10 * e ** 2)
    assert np.all(np.abs(En.barrier_d1(below, DH)) < 10 * e)
    assert np.all(np.abs(En.barrier_d2(below, DH)) < 10 * e / DH)
    beyond = DH * np.array([1.0, 1.5])
    assert np.all(En.barrier(beyond, DH) == 0) and np.all(En.barrier_d1(beyond, DH) == 0)


def test_contact_gradient_matches_central_differences():
    pad, ind, y = _pair_setup(1)
    pairs = BP.candidates(pad.rest, y, pad, ind, 2 * DH)
    x = pad.rest
    E, g, _, _ = En.contact(pairs, x, y, pad, ind)
    assert E > 0
    h = 1e-11
    worst = 0.0
    for v in np.unique(En.pair_geometry(pairs, x, y, pad, ind)[1]):
        if v < 0:
            continue
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += h
            xm[v, c] -= h
            fd = (En.contact(pairs, xp, y, pad, ind)[0] - En.contact(pairs, xm, y, pad, ind)[0]) / (2 * h)
            worst = max(worst, abs(fd - g[v, c]))
    assert worst < 1e-5 * np.abs(g).max()


def test_contact_line_curvature_matches_fd_of_gradient():
    pad, ind, y = _pair_setup(2)
    pairs = BP.candidates(pad.rest, y, pad, ind, 2 * DH)
    x = pad.rest
    rng = np.random.default_rng(3)
    p = rng.normal(size=x.shape) * (pad.free[:, None])
    j = En.contact_line(pairs, x, p, y, pad, ind)
    _, g, _, _ = En.contact(pairs, x, y, pad, ind)
    assert float(j.d) == pytest.approx(float(np.sum(g * p)), rel=1e-9)
    h = 1e-12
    _, gp, _, _ = En.contact(pairs, x + h * p, y, pad, ind)
    _, gm, _, _ = En.contact(pairs, x - h * p, y, pad, ind)
    assert float(j.dd) == pytest.approx(float(np.sum((gp - gm) * p)) / (2 * h), rel=1e-5)


def test_gauss_newton_block_exact_for_face_contact():
    """A gel vertex facing a fixed triangle's interior: grad^2 d = 0, so the
    Gauss-Newton block equals the exact Hessian block."""
    pd, pad = tiny_pad()
    v = int(np.argmax(pad.rest[:, 2] + 1e-9 * pad.rest[:, 0]))
    X = pad.rest[v]
    ind = G.build_indenter(np.array([[X[0] - 1e-3, X[1] - 1e-3, 0.0], [X[0] + 2e-3, X[1] - 1e-3, 0.0],
                                     [X[0] - 1e-3, X[1] + 2e-3, 0.0]]), np.array([[0, 1, 2]]))
    y = ind.verts.copy()
    y[:, 2] = X[2] + 0.4 * DH
    y[1, 2] += 0.1 * DH                       # tilt the plane
    pairs = np.array([[0, v, 0]])
    _, _, blk, _ = En.contact(pairs, pad.rest, y, pad, ind)
    fr = En.Frame(pad, ind, pad.rest, pad.rest, y, y, En.friction_lag(pairs, pad.rest, y, pad, ind))
    _, H = NW._pair_hessians(fr, pad.rest, 0.0, pairs)
    assert np.abs(H[0, 0, :, 0, :] - blk[v]).max() < 1e-8 * np.abs(blk[v]).max()


# ---------------------------------------------------------------------------
# friction


def test_mollifier_is_c1_at_eps():
    eps = 1e-5
    assert En.mollifier(np.array([0.0]), eps)[0] == pytest.approx(eps / 3)
    lo, hi = eps * (1 - 1e-9), eps * (1 + 1e-9)
    assert En.mollifier(np.array([lo]), eps)[0] == pytest.approx(En.mollifier(np.array([hi]), eps)[0], rel=1e-8)
    h = eps * 1e-6
    d_lo = (En.mollifier(np.array([eps - h]), eps) - En.mollifier(np.array([eps - 2 * h]), eps))[0] / h
    d_hi = (En.mollifier(np.array([eps + 2 * h]), eps) - En.mollifier(np.array([eps + h]), eps))[0] / h
    assert d_lo == pytest.approx(1.0, abs=1e-5) and d_hi == pytest.approx(1.0, abs=1e-9)
    s = np.linspace(1e-9, 2 * eps, 7)
    ds = 1e-12
    fd = (En.mollifier(s + ds, eps) - En.mollifier(s - ds, eps)) / (2 * ds)
    assert np.allclose(En.mollifier_d1_over_s(s, eps) * s, fd, rtol=1e-5)


def _friction_setup(seed=4):
    pad, ind, y = _pair_setup(seed)
    pad.mu_f = 0.5
    pairs = BP.candidates(pad.rest, y, pad, ind, 2 * DH)
    lag = En.friction_lag(pairs, pad.rest, y, pad, ind)
    assert lag["lam"].size > 0 and np.all(lag["lam"] > 0)
    rng = np.random.default_rng(seed)
    y2 = y + np.array([0.2, -0.1, 0.0]) * DH
    x = pad.rest + rng.normal(size=pad.rest.shape) * 0.1 * pad.eps_v * pad.free[:, None]
    return pad, ind, lag, x, y, y2


@pytest.mark.parametrize("seed", [4, 7])
def test_friction_lag_carries_the_barrier_forces(seed):
    """R13's lag: each pair's lagged normal force lambda_n = -kappa m b'(d),
    applied along its normal with its closest-point weights, reproduces the
    contact gradient at the frame start on every gel vertex. Where no
    edge-edge pair is inside its mollifier band (m = 1, m' = 0) the two are
    the same vector field: a lag built with the wrong sign, without kappa or
    from the wrong side's weights fails it."""
    pad, ind, y = _pair_setup(seed)
    pad.mu_f = 0.5
    x = pad.rest
    pairs = BP.candidates(x, y, pad, ind, 2 * DH)
    d, _, (ty, gid, iid) = En.distances(pairs, x, y, pad, ind)
    act = d < pad.dhat
    P = En._slot_positions(gid[act], iid[act], x, y)
    c = En.edge_cross_sq(P)
    eps = En.ee_mollifier_eps(ty[act], gid[act], iid[act], pad, ind)
    assert np.all((eps == 0) | (c >= eps))          # no pair inside the mollifier band here
    lag = En.friction_lag(pairs, x, y, pad, ind)
    assert lag["lam"].size == int(act.sum()) > 0
    g_lag = np.zeros_like(x)
    for k in range(lag["lam"].size):
        for sl in range(4):
            v = lag["gid"][k, sl]
            if v >= 0:
                g_lag[v] -= lag["lam"][k] * lag["w"][k, sl] * lag["n"][k]
    _, g, _, _ = En.contact(pairs, x, y, pad, ind)
    assert np.abs(g_lag - g).max() <= 1e-12 * np.abs(g).max()
    assert np.abs(g).max() > 0


def test_friction_gradient_matches_central_differences():
    pad, ind, lag, x, y, y2 = _friction_setup()
    E, g, _ = En.friction(lag, x, pad.rest, y2, y, pad)
    h = 1e-12
    worst = 0.0
    for v in np.unique(lag["gid"][lag["gid"] >= 0]):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += h
            xm[v, c] -= h
            fd = (En.friction(lag, xp, pad.rest, y2, y, pad)[0] - En.friction(lag, xm, pad.rest, y2, y, pad)[0]) / (2 * h)
            worst = max(worst, abs(fd - g[v, c]))
    assert worst < 1e-6 * np.abs(g).max()


def test_friction_line_and_blocks_match_exact_hessian():
    pad, ind, lag, x, y, y2 = _friction_setup(5)
    E, g, blk = En.friction(lag, x, pad.rest, y2, y, pad)
    rng = np.random.default_rng(6)
    p = rng.normal(size=x.shape) * pad.free[:, None]
    j = En.friction_line(lag, x, p, pad.rest, y2, y, pad)
    assert float(j.v) == pytest.approx(E, rel=1e-12)
    assert float(j.d) == pytest.approx(float(np.sum(g * p)), rel=1e-9)
    h = 1e-12
    _, gp, _ = En.friction(lag, x + h * p, pad.rest, y2, y, pad)
    _, gm, _ = En.friction(lag, x - h * p, pad.rest, y2, y, pad)
    assert float(j.dd) == pytest.approx(float(np.sum((gp - gm) * p)) / (2 * h), rel=1e-5)
    # diagonal block of one vertex by polarisation
    v = int(lag["gid"][0, 0])
    e = np.eye(3)

    def q(a):
        pp = np.zeros_like(x)
        pp[v] = a
        return float(En.friction_line(lag, x, pp, pad.rest, y2, y, pad).dd)
    K = np.zeros((3, 3))
    for a in range(3):
        K[a, a] = q(e[a])
    for a in range(3):
        for b in range(a + 1, 3):
            K[a, b] = K[b, a] = 0.5 * (q(e[a] + e[b]) - K[a, a] - K[b, b])
    assert np.abs(K - blk[v]).max() < 1e-6 * np.abs(K).max()
    assert np.all(np.linalg.eigvalsh(blk[v]) > -1e-12 * np.abs(blk[v]).max())


# ---------------------------------------------------------------------------
# candidate set


def test_candidates_contain_every_close_pair():
    for seed in range(3):
        pad, ind, y = _pair_setup(seed)
        r = 2 * DH
        cand = BP.candidates(pad.rest, y, pad, ind, r)
        close = BP.brute_force_close(pad.rest, y, pad, ind, r)
        cs = set(map(tuple, cand.tolist()))
        assert len(close) > 0
        assert all(tuple(c) in cs for c in close.tolist())
        # sorted lexicographically, no duplicates
        assert len(cs) == len(cand)
        assert np.all(np.diff(cand[:, 0] * 10 ** 12 + cand[:, 1] * 10 ** 6 + cand[:, 2]) > 0)


def test_non_candidates_are_farther_than_r():
    pad, ind, y = _pair_setup(7)
    r = 2 * DH
    cand = set(map(tuple, BP.candidates(pad.rest, y, pad, ind, r).tolist()))
    ap = BP.all_pairs(pad, ind)
    rest = np.array([p for p in ap.tolist() if tuple(p) not in cand])
    d, _, _ = En.distances(rest, pad.rest, y, pad, ind)
    assert d.min() > r


def test_surface_counts_of_hex_pad():
    pd, pad = tiny_pad(cells=(10, 8, 2), size=(20 * MM, 16 * MM, 4 * MM))
    # boundary vertices of an 11 x 9 x 3 lattice; two triangles per boundary quad
    assert pad.surf_verts.size == 11 * 9 * 3 - 9 * 7 * 1
    assert pad.surf_tris.shape[0] == 2 * 2 * (10 * 8 + 10 * 2 + 8 * 2)
    V, Fc, Ec = pad.surf_verts.size, pad.surf_tris.shape[0], pad.surf_edges.shape[0]
    assert V - Ec + Fc == 2                              # Euler characteristic of a closed surface
