"""Pins of oracle functions that the GPU is compared against directly:
the conservative step bound alpha_ccd of the per-pair CCD and the coupled
indenter-gel advance bound (their defining property, and exactness where
the closing speed is known) and the
candidate predicate of the set C of Eq. (ipc_energy) at its exact boundary
(inflated-AABB gaps of r and r + one float32 ulp, decided against exact
rational arithmetic)."""
from fractions import Fraction
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import broadphase as BP
from oracle import energy as En
from oracle import geometry as G
from oracle import solver as SV

from _cases import MM, small_indenter, tiny_pad

DH = 0.05 * MM
ETA = 0.9


def _frame_near_contact(seed):
    """Tiny jittered pad with a small icosphere 0.3 dhat above its top face:
    candidates of all three types, indenter fixed (s = 0)."""
    pd, pad = tiny_pad(cells=(3, 3, 1), size=(3 * MM, 3 * MM, 1 * MM), jitter=0.1, seed=seed)
    _, ind = small_indenter(radius=0.6 * MM, subdiv=1)
    ztop = pad.rest[:, 2].max()
    pose = np.array([0.3, -0.2, 0.1, 1.4 * MM, 1.6 * MM, 0.0])
    y0 = G.indenter_world(ind.verts, pose)
    pose[5] = ztop - y0[:, 2].min() + 0.3 * DH
    y = G.indenter_world(ind.verts, pose)
    x = pad.rest.astype(np.float64)
    lag = En.friction_lag(np.zeros((0, 3), np.int64), x, y, pad, ind)
    fr = En.Frame(pad, ind, x, x.copy(), y, y, lag)
    pairs = BP.candidates(x, y, pad, ind, 2 * DH)
    return fr, x, y, pairs


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ccd_bound_keeps_every_candidate_gap(seed):
    """For every alpha in (0, alpha_ccd], every candidate keeps
    d_k(x + alpha p) >= (1 - eta) d_k(x): the property the step bound of
    the line search exists for. Random directions, some pushing the gel up
    into the indenter."""
    fr, x, y, pairs = _frame_near_contact(seed)
    d0, _, _ = En.distances(pairs, x, y, fr.pad, fr.ind)
    assert len(pairs) > 0 and d0.min() > 0
    rng = np.random.default_rng(100 + seed)
    for trial in range(6):
        p = rng.normal(size=x.shape) * 1e-4
        if trial % 2:
            p[:, 2] = np.abs(p[:, 2]) * 3.0        # toward the indenter above
        a = SV.ccd_bound(fr, x, p, 0.0, pairs, ETA)
        assert np.isfinite(a) and a > 0
        for al in np.linspace(0.0, a, 17)[1:]:
            d, _, _ = En.distances(pairs, x + al * p, y, fr.pad, fr.ind)
            assert np.all(d >= (1.0 - ETA) * d0 * (1.0 - 1e-9)), (trial, al / a)


def test_ccd_bound_is_tight_for_a_rigid_approach():
    """The whole gel translating straight up at speed c: every gel
    primitive closes on the indenter at most at rate c, and the pair over a
    face closes exactly at rate c. alpha_ccd must then be eta * d_min / c,
    and at alpha_ccd the closest pair has exactly (1 - eta) of its gap
    left (a bound built from the wrong side's speeds, or off by a factor,
    fails one of the two)."""
    pad_pd, pad = tiny_pad(cells=(3, 3, 1), size=(3 * MM, 3 * MM, 1 * MM))
    # a flat horizontal indenter triangle above the pad centre: the closest
    # pairs are gel vertices under its face, with a vertical normal
    ztop = pad.rest[:, 2].max()
    gap = 0.4 * DH
    cx, cy = 1.5 * MM, 1.5 * MM
    yv = np.array([[cx - 1.2 * MM, cy - 1.2 * MM, ztop + gap], [cx + 1.3 * MM, cy - 1.1 * MM, ztop + gap],
                   [cx, cy + 1.4 * MM, ztop + gap]])
    ind = G.build_indenter(yv.astype(np.float32), np.array([[0, 2, 1]], np.int32))
    y = ind.verts.astype(np.float64)
    x = pad.rest.astype(np.float64)
    lag = En.friction_lag(np.zeros((0, 3), np.int64), x, y, pad, ind)
    fr = En.Frame(pad, ind, x, x.copy(), y, y, lag)
    pairs = BP.candidates(x, y, pad, ind, 2 * DH)
    d0, _, _ = En.distances(pairs, x, y, pad, ind)
    c = 3.0e-4
    p = np.zeros_like(x)
    p[:, 2] = c
    a = SV.ccd_bound(fr, x, p, 0.0, pairs, ETA)
    assert a == pytest.approx(ETA * d0.min() / c, rel=1e-12)
    d1, _, _ = En.distances(pairs, x + a * p, y, pad, ind)
    k = int(np.argmin(d0))
    assert d1[k] == pytest.approx((1.0 - ETA) * d0[k], rel=1e-6)
    assert np.all(d1 >= (1.0 - ETA) * d0 * (1.0 - 1e-9))


# ---------------------------------------------------------------------------
# the coupled indenter-gel advance bound (R11)


def _moving_frame(seed):
    """The near-contact frame with the indenter moving over the frame on its
    per-vertex straight path: a small rotation and a translation down and
    sideways, so dy differs per vertex."""
    fr, x, y, pairs = _frame_near_contact(seed)
    rng = np.random.default_rng(200 + seed)
    ind = fr.ind
    c = y.mean(axis=0)
    ang = rng.uniform(-0.05, 0.05, 3)
    th = np.linalg.norm(ang)
    k = ang / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    R = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    y_n = (y - c) @ R.T + c + np.array([0.3, -0.2, -1.5]) * DH
    fr2 = En.Frame(fr.pad, ind, x, x.copy(), y, y_n, fr.lag)
    return fr2, x, y, y_n, pairs


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_advance_bound_keeps_every_candidate_gap(seed):
    """For every advance sigma in (0, ds], ds the bound of the coupled
    advance at path parameter s (gel along w, indenter on its straight
    per-vertex path), every candidate keeps
    d_k(x + sigma w, y(s + sigma)) >= (1 - eta) d_k(x, y(s)): the property
    the substep bound exists for. Random gel motions, some pushing the gel
    up into the indenter, and the gel held (w = 0)."""
    fr, x, y_t, y_n, pairs = _moving_frame(seed)
    dy = y_n - y_t
    s = 0.3
    d0, _, _ = En.distances(pairs, x, fr.y(s), fr.pad, fr.ind)
    assert len(pairs) > 0 and d0.min() > 0
    rng = np.random.default_rng(300 + seed)
    for trial in range(5):
        w = rng.normal(size=x.shape) * 0.5 * DH
        if trial % 2:
            w[:, 2] = np.abs(w[:, 2]) * 2.0
        if trial == 4:
            w[:] = 0.0
        ds = SV.advance_bound(fr, x, s, pairs, w, dy, ETA)
        assert np.isfinite(ds) and ds > 0
        for sg in np.linspace(0.0, ds, 17)[1:]:
            d, _, _ = En.distances(pairs, x + sg * w, y_t + (s + sg) * dy, fr.pad, fr.ind)
            assert np.all(d >= (1.0 - ETA) * d0 * (1.0 - 1e-9)), (trial, sg / ds)


def test_advance_bound_is_tight_for_opposed_translations():
    """The gel translating up at speed a and the indenter straight down at
    speed b: every primitive pair closes at most at a + b, the pairs under
    the indenter's face exactly so. The bound must be eta d_min / (a + b),
    and there the closest pair has exactly (1 - eta) of its gap left (a
    bound that drops one side's motion, or adds them with the wrong sign,
    fails)."""
    pad_pd, pad = tiny_pad(cells=(3, 3, 1), size=(3 * MM, 3 * MM, 1 * MM))
    ztop = pad.rest[:, 2].max()
    gap = 0.4 * DH
    cx, cy = 1.5 * MM, 1.5 * MM
    yv = np.array([[cx - 1.2 * MM, cy - 1.2 * MM, ztop + gap], [cx + 1.3 * MM, cy - 1.1 * MM, ztop + gap],
                   [cx, cy + 1.4 * MM, ztop + gap]])
    ind = G.build_indenter(yv.astype(np.float32), np.array([[0, 2, 1]], np.int32))
    y_t = ind.verts.astype(np.float64)
    a_up, b_down = 1.0e-5, 2.5e-5
    y_n = y_t - np.array([0.0, 0.0, b_down])
    x = pad.rest.astype(np.float64)
    lag = En.friction_lag(np.zeros((0, 3), np.int64), x, y_t, pad, ind)
    fr = En.Frame(pad, ind, x, x.copy(), y_t, y_n, lag)
    pairs = BP.candidates(x, y_t, pad, ind, 2 * DH)
    d0, _, _ = En.distances(pairs, x, y_t, pad, ind)
    w = np.zeros_like(x)
    w[:, 2] = a_up
    dy = y_n - y_t
    ds = SV.advance_bound(fr, x, 0.0, pairs, w, dy, ETA)
    assert ds == pytest.approx(ETA * d0.min() / (a_up + b_down), rel=1e-12)
    d1, _, _ = En.distances(pairs, x + ds * w, y_t + ds * dy, pad, ind)
    k = int(np.argmin(d0))
    assert d1[k] == pytest.approx((1.0 - ETA) * d0[k], rel=1e-6)
    assert np.all(d1 >= (1.0 - ETA) * d0 * (1.0 - 1e-9))


# ---------------------------------------------------------------------------
# the candidate predicate at its boundary


def _f32(v):
    return np.float32(v)


def _boundary_value(base, r, up):
    """float32 coordinates L next to base + r (base float32, r float64):
    the largest L with L - base <= r (exactly) or, with ``up``, the smallest
    L with L - base > r."""
    B, R = Fraction(float(base)), Fraction(float(r))
    L = _f32(float(base) + float(r))
    while Fraction(float(L)) - B > R:
        L = np.nextafter(L, np.float32(-np.inf))
    while Fraction(float(np.nextafter(L, np.float32(np.inf)))) - B <= R:
        L = np.nextafter(L, np.float32(np.inf))
    return np.nextafter(L, np.float32(np.inf)) if up else L


def _exact_overlap(gp, ip, r):
    """Exact rational inflated-AABB predicate for one pair of primitives."""
    R = Fraction(float(r))
    for a in range(3):
        glo = min(Fraction(float(v[a])) for v in gp)
        ghi = max(Fraction(float(v[a])) for v in gp)
        ilo = min(Fraction(float(v[a])) for v in ip)
        ihi = max(Fraction(float(v[a])) for v in ip)
        if not (glo - R <= ihi and ilo <= ghi + R):
            return False
    return True


def _tiny_models(xg, yi):
    """A gel surface of one triangle (its 3 vertices and 3 edges) and an
    indenter of one triangle (3 vertices, 3 edges)."""
    pad = SimpleNamespace(surf_verts=np.array([0, 1, 2]), surf_tris=np.array([[0, 1, 2]]),
                          surf_edges=np.array([[0, 1], [0, 2], [1, 2]]))
    ind = SimpleNamespace(tris=np.array([[0, 1, 2]]), edges=np.array([[0, 1], [0, 2], [1, 2]]),
                          verts=yi)
    return pad, ind


def _exact_set(xg, yi, pad, ind, r):
    out = []
    for i in pad.surf_verts:
        for j in range(ind.tris.shape[0]):
            if _exact_overlap([xg[i]], yi[ind.tris[j]], r):
                out.append((0, int(i), j))
    for i in range(pad.surf_tris.shape[0]):
        for j in range(yi.shape[0]):
            if _exact_overlap(xg[pad.surf_tris[i]], [yi[j]], r):
                out.append((1, i, j))
    for i in range(pad.surf_edges.shape[0]):
        for j in range(ind.edges.shape[0]):
            if _exact_overlap(xg[pad.surf_edges[i]], yi[ind.edges[j]], r):
                out.append((2, i, j))
    return sorted(out)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("side", [1, -1])
@pytest.mark.parametrize("r", [(DH + DH) * (1.0 + 1e-6), 2.0 ** -13])
def test_candidate_predicate_at_exact_boundary(axis, side, r):
    """Indenter placed so that its box's gap to the gel box along one axis
    is r (within float32 placement: the last float32 at or below it) or one
    float32 ulp beyond: the pairs across that gap are candidates in the
    first case and not in the second, exactly as rational arithmetic
    decides. With r = 2^-13 the gap is r exactly (float32 coordinates hold
    it), so the comparison's equality case is taken too. An over-inclusive
    predicate (inflation 2r, or r on both boxes) or a strict inequality
    fails here."""
    xg = np.array([[1.25e-3, 2.5e-3, 1.0e-3], [1.75e-3, 2.625e-3, 1.125e-3], [1.5e-3, 3.0e-3, 1.0625e-3]],
                  dtype=np.float32)
    base = (xg[:, axis].max() if side > 0 else xg[:, axis].min())
    for up in (False, True):
        # a triangle overlapping the gel box on the other axes, lying beyond it on this axis
        yi = np.array([[1.3e-3, 2.55e-3, 1.05e-3], [1.7e-3, 2.6e-3, 1.1e-3], [1.5e-3, 2.9e-3, 1.06e-3]],
                      dtype=np.float32)
        if side > 0:
            L = _boundary_value(base, r, up)
            shift = [L, L + _f32(1e-5), L + _f32(2e-5)]
        else:
            L = -_boundary_value(-base, r, up)       # mirrored: base - L <= r
            shift = [L, L - _f32(1e-5), L - _f32(2e-5)]
        yi[:, axis] = np.array(shift, dtype=np.float32)
        pad, ind = _tiny_models(xg, yi)
        got = BP.candidates(xg.astype(np.float64), yi.astype(np.float64), pad, ind, r)
        want = _exact_set(xg, yi, pad, ind, r)
        assert [tuple(t) for t in got.tolist()] == want, (axis, side, up)
        # the vertex-triangle pair whose gap is the boundary itself
        gv = int(np.argmax(xg[:, axis])) if side > 0 else int(np.argmin(xg[:, axis]))
        assert ((0, gv, 0) in want) == (not up)


# ---------------------------------------------------------------------------
# the parallel-edge mollifier of the edge-edge barrier


def _parallel_edge_scene(angle, gap=0.3 * DH):
    """Tiny pad and a one-triangle indenter whose lower edge lies ``gap``
    above the pad's top face, turned by ``angle`` (rad) from the x-aligned
    top edges of the pad in the horizontal plane: edge-edge candidates
    between the lower edge and x-aligned gel edges are parallel at
    angle = 0."""
    pd, pad = tiny_pad(cells=(3, 3, 1), size=(3 * MM, 3 * MM, 1 * MM))
    ztop = pad.rest[:, 2].max()
    c, s = np.cos(angle), np.sin(angle)
    y0 = np.array([1.5 * MM, 1.0 * MM, ztop + gap])
    yv = np.array([y0 - 1.2 * MM * np.array([c, s, 0.0]), y0 + 1.3 * MM * np.array([c, s, 0.0]),
                   y0 + np.array([0.0, 0.0, 0.8 * MM])])
    ind = G.build_indenter(yv, np.array([[0, 1, 2]], np.int32))
    y = ind.verts.copy()
    x = pad.rest.astype(np.float64)
    pairs = BP.candidates(x, y, pad, ind, 2 * DH)
    return pad, ind, x, y, pairs


def test_ee_mollifier_shape():
    """m(0) = 0, m(eps) = 1 with m'(eps) = 0 (C^1 join to the constant 1),
    monotone on [0, eps]; m' matches a central difference."""
    eps = np.array([1.0])
    cs = np.linspace(0.0, 2.0, 41)
    m = np.array([En.ee_mollifier(np.array([c]), eps)[0] for c in cs])
    assert m[0] == 0.0 and m[20] == pytest.approx(1.0) and np.all(m[20:] == 1.0)
    assert np.all(np.diff(m[:21]) > 0)
    for c in (0.3, 0.7, 0.9999):
        h = 1e-6
        fd = (En.ee_mollifier(np.array([c + h]), eps)[0] - En.ee_mollifier(np.array([c - h]), eps)[0]) / (2 * h)
        assert En.ee_mollifier_d1(np.array([c]), eps)[0] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    assert En.ee_mollifier_d1(np.array([1.0 - 1e-12]), eps)[0] == pytest.approx(0.0, abs=1e-9)


@pytest.mark.parametrize("angle", [0.0, 2e-3, 0.2])
def test_mollified_contact_gradient_matches_differences(angle):
    """Gradient of kappa sum m(c) b(d) against central differences of the
    energy at near-parallel (inside the mollifier band), parallel and
    clearly crossing edge-edge configurations, with random gel offsets."""
    pad, ind, x, y, pairs = _parallel_edge_scene(angle)
    assert np.any(pairs[:, 0] == 2)
    rng = np.random.default_rng(5)
    x = x + rng.normal(size=x.shape) * 0.02 * DH
    E, g, _, _ = En.contact(pairs, x, y, pad, ind)
    near = np.unique(np.concatenate([BP.candidates(x, y, pad, ind, DH)[:, 1:2].ravel()]))
    verts = np.unique(pad.surf_edges[pairs[pairs[:, 0] == 2, 1]].ravel())[:12]
    h = 1e-11
    for v in verts:
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += h
            xm[v, c] -= h
            fd = (En.contact(pairs, xp, y, pad, ind)[0] - En.contact(pairs, xm, y, pad, ind)[0]) / (2 * h)
            assert g[v, c] == pytest.approx(fd, rel=1e-4, abs=1e-6 * np.abs(g).max())
    del near


def test_mollified_edge_edge_term_is_smooth_through_parallel():
    """Along a line that turns an edge-edge pair through exactly parallel
    (the configuration a pressed edge settles into), the unmollified
    barrier has a kink; the mollified one has equal one-sided slopes, and
    its line derivatives (Taylor arithmetic) match differences of the
    energy."""
    pad, ind, x, y, pairs = _parallel_edge_scene(0.0)
    ee = pairs[pairs[:, 0] == 2]
    ty, gid, iid = En.pair_geometry(ee, x, y, pad, ind)
    P = En._slot_positions(gid, iid, x, y)
    d, _ = En.slot_distances(ty, P)
    # the closest x-aligned gel edge: parallel to the indenter edge above it
    ex = np.abs(P[:, 1, 0] - P[:, 0, 0]) > 0.9 * np.linalg.norm(P[:, 1] - P[:, 0], axis=1)
    k = int(np.argmin(np.where(ex, d, np.inf)))
    pair = ee[k:k + 1]
    a, b = pad.surf_edges[pair[0, 1]]
    # tilt the gel edge about its midpoint in its vertical plane: one end
    # rises towards the indenter edge above it whichever way it turns
    p = np.zeros_like(x)
    n = np.array([0.0, 0.0, 1.0])
    p[a], p[b] = -0.5 * n * 1e-3, 0.5 * n * 1e-3
    eps = En.ee_mollifier_eps(ty[k:k + 1], gid[k:k + 1], iid[k:k + 1], pad, ind)

    def raw(al):
        P1 = En._slot_positions(gid[k:k + 1], iid[k:k + 1], x + al * p, y)
        return float(En.barrier(En.slot_distances(ty[k:k + 1], P1)[0], pad.dhat)[0])

    def moll(al):
        P1 = En._slot_positions(gid[k:k + 1], iid[k:k + 1], x + al * p, y)
        return float(En.pair_barrier(ty[k:k + 1], P1, eps, pad.dhat)[0])

    def kink(f, h):      # right slope minus left slope at 0
        return (f(h) - f(0)) / h - (f(0) - f(-h)) / h

    # a kink keeps its slope jump as h shrinks; a C^1 function's shrinks with h
    h = 1e-3
    assert abs(kink(raw, h)) > 0.5 * abs(raw(h) - raw(0)) / h
    assert kink(raw, h / 10) == pytest.approx(kink(raw, h), rel=0.05)
    assert abs(kink(moll, h / 10)) < 0.15 * abs(kink(moll, h))
    assert abs(kink(moll, h / 100)) < 0.02 * abs(kink(moll, h))
    # Taylor-arithmetic line derivatives of the whole contact term at a
    # nearby non-parallel point match differences of the energy
    x1 = x + 1e-2 * p           # the raised end still 2/3 of the gap away
    jet = En.contact_line(pairs, x1, p, y, pad, ind)
    q = 1e-5
    e = [En.contact(pairs, x1 + t * p, y, pad, ind)[0] for t in (-q, 0.0, q)]
    assert jet.v == pytest.approx(e[1], rel=1e-12)
    assert jet.d == pytest.approx((e[2] - e[0]) / (2 * q), rel=1e-4)
    assert jet.dd == pytest.approx((e[2] - 2 * e[1] + e[0]) / q ** 2, rel=1e-3)
