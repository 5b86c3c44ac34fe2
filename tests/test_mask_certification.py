"""The float32 candidate masks of the pair passes (pt_mask / ee_mask in
csrc/device_math.cuh), emulated in numpy float32, against the full float64
closest-feature search.

The kernels run the float64 point-triangle / edge-edge search only over the
candidates the float32 pass marks; the mask must hold every candidate that
can win the float64 search, so that the masked search returns the full
search's feature. The emulation perturbs float32 slot positions by up to one
ulp (the kernels' bound allows 8 units of 2^-24 of the largest coordinate)
and draws adversarial configurations: points within 1e-6 (relative) of
triangle edges and vertices, edge pairs crossing near their ends or nearly
parallel, gaps from 1e-8 to 1e-4 m at coordinates up to 2 cm. It mirrors the
kernels' formulas (without FMA contraction, which the margins cover).
"""
import numpy as np
import pytest

f32 = np.float32
EX_UNITS = f32(4.76837158203125e-7)      # 8 x 2^-24: the kernels' bound per unit coordinate
REL = f32(9.5367431640625e-7)            # 2^-20: the distance's own rounding
AR = f32(1.9073486328125e-6)             # 2^-19: the edge-edge solve's cancellation term


def dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def cross(a, b):
    return np.array([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]],
                    dtype=a.dtype)


def seg_param(P, A, B):
    """Squared distance of P to segment AB (clamped parameter), in P's type."""
    T = P.dtype.type
    e = B - A
    ee = dot(e, e)
    t = T(min(max(dot(P - A, e) / ee, 0), 1)) if ee > 0 else T(0)
    r = P - (A + t * e)
    return dot(r, r)


def pt_full(P, A, B, C):
    """Full float64 point-triangle search: (winning candidate, distance)."""
    v0, v1, v2 = B - A, C - A, P - A
    d00, d01, d11, d20, d21 = dot(v0, v0), dot(v0, v1), dot(v1, v1), dot(v2, v0), dot(v2, v1)
    den = d00 * d11 - d01 * d01
    l1 = (d11 * d20 - d01 * d21) / den
    l2 = (d00 * d21 - d01 * d20) / den
    l0 = 1 - l1 - l2
    best, k = np.inf, -1
    if l0 >= 0 and l1 >= 0 and l2 >= 0 and den > 0:
        n = cross(v0, v1)
        s = dot(v2, n)
        best, k = s * s / dot(n, n), 0
    for j, (X, Y) in enumerate(((A, B), (B, C), (C, A))):
        dj = seg_param(P, X, Y)
        if k < 0 or dj < best:
            best, k = dj, j + 1
    return k, np.sqrt(best)


def _edge_mask(de, ex, mask):
    """Point-segment candidates within twice the error bound of the best."""
    r = np.sqrt(min(de))
    lim = r + f32(2) * (f32(6) * ex + REL * r)
    for j, dj in enumerate(de):
        if dj <= lim * lim:
            mask |= 2 << j
    return mask


def pt_mask(P, A, B, C, ex):
    """float32 candidate mask of a point-triangle pair (pt_mask)."""
    v0, v1, v2 = B - A, C - A, P - A
    d00, d01, d11, d20, d21 = dot(v0, v0), dot(v0, v1), dot(v1, v1), dot(v2, v0), dot(v2, v1)
    den = d00 * d11 - d01 * d01
    l1 = (d11 * d20 - d01 * d21) / den
    l2 = (d00 * d21 - d01 * d20) / den
    l0 = f32(1) - l1 - l2
    face = -1
    if den > f32(1e-6) * d00 * d11:
        nn, tol, v3 = np.sqrt(den), f32(16) * ex, v1 - v0
        m = (l0 * nn / np.sqrt(dot(v3, v3)), l1 * nn / np.sqrt(d11), l2 * nn / np.sqrt(d00))
        if min(m) >= tol:
            face = 1
        elif min(m) <= -tol:
            face = 0
    if face == 1:
        return 1
    de = [seg_param(P, A, B), seg_param(P, B, C), seg_param(P, C, A)]
    return _edge_mask(de, ex, 1 if face < 0 else 0)


def ee_full(P0, P1, Q0, Q1):
    """Full float64 edge-edge search: (winning candidate, distance)."""
    u, v, w = P1 - P0, Q1 - Q0, P0 - Q0
    a, b, c, dd, e = dot(u, u), dot(u, v), dot(v, v), dot(u, w), dot(v, w)
    D = a * c - b * b
    best, k = np.inf, -1
    if D > 1e-12 * a * c:
        s = (b * e - c * dd) / D
        t = (a * e - b * dd) / D
        if 0 <= s <= 1 and 0 <= t <= 1:
            r = w + s * u - t * v
            best, k = dot(r, r), 0
    for j, (X, A, B) in enumerate(((P0, Q0, Q1), (P1, Q0, Q1), (Q0, P0, P1), (Q1, P0, P1))):
        dj = seg_param(X, A, B)
        if k < 0 or dj < best:
            best, k = dj, j + 1
    return k, np.sqrt(best)


def ee_mask(P0, P1, Q0, Q1, ex):
    """float32 candidate mask of an edge-edge pair (ee_mask)."""
    u, v, w = P1 - P0, Q1 - Q0, P0 - Q0
    a, b, c, dd, e = dot(u, u), dot(u, v), dot(v, v), dot(u, w), dot(v, w)
    D = a * c - b * b
    inter = -1
    if D > f32(1e-12) * a * c:
        s = (b * e - c * dd) / D
        t = (a * e - b * dd) / D
        if D > f32(1e-4) * a * c:
            sD, cond = np.sqrt(D), a * c * (f32(1) / D)
            ar = AR * cond * (f32(1) + np.sqrt(dot(w, w) / min(a, c)))
            ms = f32(16) * ex * np.sqrt(c) / sD + ar
            mt = f32(16) * ex * np.sqrt(a) / sD + ar
            if ms <= s <= f32(1) - ms and mt <= t <= f32(1) - mt:
                inter = 1
            elif s < -ms or s > f32(1) + ms or t < -mt or t > f32(1) + mt:
                inter = 0
    if inter == 1:
        return 1
    de = [seg_param(P0, Q0, Q1), seg_param(P1, Q0, Q1), seg_param(Q0, P0, P1), seg_param(Q1, P0, P1)]
    return _edge_mask(de, ex, 1 if inter < 0 else 0)


def to32(X, rng):
    """float32 positions within ~2 ulp of the float64 ones."""
    Xf = X.astype(f32)
    ul = np.spacing(np.abs(Xf)).astype(f32)
    return (Xf + ul * rng.integers(-1, 2, size=X.shape).astype(f32)).astype(f32)


@pytest.mark.parametrize("seed", [0, 1])
def test_masks_keep_the_float64_winner(seed, n=10000):
    rng = np.random.default_rng(seed)
    misses, multi = 0, 0
    for it in range(n):
        base = rng.uniform(0.0, 0.02, 3)
        L = rng.choice([1e-4, 2e-4, 5e-4, 2e-3])
        if it % 2 == 0:
            A = base
            B = base + rng.normal(size=3) * L
            C = base + rng.normal(size=3) * L
            n_ = np.cross(B - A, C - A)
            n_ /= np.linalg.norm(n_)
            mode = rng.integers(0, 4)
            bc = rng.dirichlet([1, 1, 1])
            if mode == 1:
                bc[rng.integers(0, 3)] = rng.normal() * 1e-6
            if mode == 2:
                bc = np.zeros(3)
                bc[rng.integers(0, 3)] = 1
                bc += rng.normal(size=3) * 1e-6
            q = bc[0] * A + bc[1] * B + bc[2] * C
            dist = 10 ** rng.uniform(-8, -4)
            P = q + n_ * dist * rng.choice([-1, 1]) + (rng.normal(size=3) * 1e-7 if mode == 3 else 0)
            k64, _ = pt_full(P, A, B, C)
            X32 = to32(np.stack([P, A, B, C]), rng)
            ex = EX_UNITS * f32(np.abs(X32).max())
            m = pt_mask(*X32, ex)
        else:
            P0 = base
            P1 = base + rng.normal(size=3) * L
            u = P1 - P0
            dirv = rng.normal(size=3)
            if rng.random() < 0.3:
                dirv = u / np.linalg.norm(u) + rng.normal(size=3) * 10 ** rng.uniform(-5, -1)
            s0 = rng.choice([rng.uniform(0, 1), rng.normal() * 1e-6, 1 + rng.normal() * 1e-6])
            t0 = rng.choice([rng.uniform(0, 1), rng.normal() * 1e-6, 1 + rng.normal() * 1e-6])
            nrm = np.cross(u, dirv)
            nrm /= np.linalg.norm(nrm)
            dist = 10 ** rng.uniform(-8, -4)
            v = dirv / np.linalg.norm(dirv) * rng.choice([1e-4, 2e-4, 5e-4])
            Q0 = P0 + s0 * u + nrm * dist - t0 * v
            Q1 = Q0 + v
            k64, _ = ee_full(P0, P1, Q0, Q1)
            X32 = to32(np.stack([P0, P1, Q0, Q1]), rng)
            ex = EX_UNITS * f32(np.abs(X32).max())
            m = ee_mask(*X32, ex)
        multi += bin(m).count("1") > 1
        misses += not (m >> k64) & 1
    assert misses == 0
    # the draw is adversarial: many cases sit within the margins
    assert multi > n // 10
