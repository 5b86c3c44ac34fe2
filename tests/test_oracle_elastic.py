"""Pins of the oracle's elasticity and inertia against closed forms, finite
differences and the Taylor-arithmetic derivatives of the energy itself."""
import numpy as np
import pytest

from oracle import energy as En
from oracle import geometry as G
from oracle import newton as NW
from oracle import taylor as T

from _cases import MM, tiny_pad


def _lin_energy(x, pad):
    return En.elastic(x, pad, blocks=False)[0]


def test_rest_state_is_stress_free():
    _, pad = tiny_pad()
    E, g, _ = En.elastic(pad.rest, pad)
    assert abs(E) < 1e-20 * pad.g_ref * pad.dhat
    assert np.abs(g).max() < 1e-12 * pad.g_ref          # rounding of F = Ds Dm^-1 only


def test_lame_parameters():
    mu, lam = G.lame(0.3e6, 0.45)
    assert mu == pytest.approx(0.3e6 / 2.9)
    assert lam == pytest.approx(0.3e6 * 0.45 / (1.45 * 0.1))
    assert lam / mu == pytest.approx(2 * 0.45 / (1 - 2 * 0.45))


@pytest.mark.parametrize("s", [0.9, 0.97, 1.05])
def test_uniform_compression_patch(s):
    """Affine F = diag(1, 1, s): interior vertices feel no force, the energy
    is V_tot * Psi(F) (closed form) and the summed z-gradient on the top
    face is h^2 P_zz A_top with P_zz = mu (s - 1/s) + lam ln(s) / s."""
    pd, pad = tiny_pad(cells=(3, 3, 2), size=(3 * MM, 3 * MM, 2 * MM))
    F = np.diag([1.0, 1.0, s])
    x = pad.rest @ F.T
    E, g, _ = En.elastic(x, pad, blocks=False)
    mu, lam = pad.mu, pad.lam
    psi = 0.5 * mu * (2 + s * s - 3) - mu * np.log(s) + 0.5 * lam * np.log(s) ** 2
    h2 = pad.h ** 2
    X = pad.rest
    lx, ly, lz = X.max(axis=0) - X.min(axis=0)           # float32 rest extents
    assert E == pytest.approx(h2 * lx * ly * lz * psi, rel=1e-10)
    interior = np.all((X > 1e-12) & (X < X.max(axis=0) - 1e-12), axis=1)
    assert interior.sum() > 0
    assert np.abs(g[interior]).max() < 1e-12 * np.abs(g).max()
    top = X[:, 2] == X[:, 2].max()
    Pzz = mu * (s - 1 / s) + lam * np.log(s) / s
    assert g[top, 2].sum() == pytest.approx(h2 * Pzz * lx * ly, rel=1e-10)


def test_random_affine_interior_equilibrium():
    pd, pad = tiny_pad(cells=(3, 3, 2), size=(3 * MM, 3 * MM, 2 * MM))
    rng = np.random.default_rng(1)
    F = np.eye(3) + 0.05 * rng.normal(size=(3, 3))
    x = pad.rest @ F.T
    _, g, _ = En.elastic(x, pad, blocks=False)
    X = pad.rest
    interior = np.all((X > 1e-12) & (X < np.array(pd.size) - 1e-12), axis=1)
    assert np.abs(g[interior]).max() < 1e-11 * np.abs(g).max()


def test_gradient_matches_central_differences():
    _, pad = tiny_pad(jitter=0.1)
    rng = np.random.default_rng(2)
    x = pad.rest + 2e-5 * rng.normal(size=pad.rest.shape)
    _, g, _ = En.elastic(x, pad, blocks=False)
    h = 1e-9
    fd = np.zeros_like(x)
    for i in range(x.shape[0]):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            fd[i, c] = (_lin_energy(xp, pad) - _lin_energy(xm, pad)) / (2 * h)
    assert np.abs(fd - g).max() < 1e-6 * np.abs(g).max()


def test_line_jet_matches_gradient_and_fd_curvature():
    _, pad = tiny_pad(jitter=0.1)
    rng = np.random.default_rng(3)
    x = pad.rest + 3e-5 * rng.normal(size=pad.rest.shape)
    p = rng.normal(size=x.shape)
    E, g, _ = En.elastic(x, pad, blocks=False)
    jet = En.elastic_line(x, p, pad)
    assert float(jet.v) == pytest.approx(E, rel=1e-12)
    assert float(jet.d) == pytest.approx(float(np.sum(g * p)), rel=1e-10)
    h = 1e-7
    _, gp, _ = En.elastic(x + h * p, pad, blocks=False)
    _, gm, _ = En.elastic(x - h * p, pad, blocks=False)
    assert float(jet.dd) == pytest.approx(float(np.sum((gp - gm) * p)) / (2 * h), rel=1e-6)


def _jet_block(x, pad, i):
    """Diagonal 3x3 Hessian block of vertex i by polarisation of Jets."""
    def q(v):
        p = np.zeros_like(x)
        p[i] = v
        return float(En.elastic_line(x, p, pad).dd)
    e = np.eye(3)
    K = np.zeros((3, 3))
    for a in range(3):
        K[a, a] = q(e[a])
    for a in range(3):
        for b in range(a + 1, 3):
            K[a, b] = K[b, a] = 0.5 * (q(e[a] + e[b]) - K[a, a] - K[b, b])
    return K


def test_diagonal_blocks_are_exact_hessian_blocks():
    _, pad = tiny_pad(jitter=0.1)
    rng = np.random.default_rng(4)
    x = pad.rest + 5e-5 * rng.normal(size=pad.rest.shape)
    _, _, blk = En.elastic(x, pad)
    for i in range(0, x.shape[0], 3):
        K = _jet_block(x, pad, i)
        assert np.abs(K - blk[i]).max() < 1e-9 * np.abs(K).max()


def test_exact_tet_hessian_matches_jet():
    _, pad = tiny_pad(jitter=0.1)
    rng = np.random.default_rng(5)
    x = pad.rest + 5e-5 * rng.normal(size=pad.rest.shape)
    He = NW.elastic_hessian_blocks(x, pad)
    p = rng.normal(size=x.shape)
    pt = p[pad.tets]                                    # [T, 4, 3]
    q = float(np.einsum("tia,tiajc,tjc->", pt, He, pt))
    assert q == pytest.approx(float(En.elastic_line(x, p, pad).dd), rel=1e-10)


def test_inverted_tet_has_infinite_energy():
    _, pad = tiny_pad()
    x = pad.rest.copy()
    t0 = pad.tets[0]
    x[t0[3]] = x[t0[0]] - (x[t0[3]] - x[t0[0]])        # reflect one corner through another
    assert not np.isfinite(En.elastic(x, pad)[0])


def test_lumped_mass_sums_to_total():
    pd, pad = tiny_pad()
    lx, ly, lz = pad.rest.max(axis=0) - pad.rest.min(axis=0)
    assert pad.mass.sum() == pytest.approx(1100.0 * lx * ly * lz, rel=1e-12)


def test_inertia_line():
    _, pad = tiny_pad()
    rng = np.random.default_rng(6)
    x = pad.rest + rng.normal(size=pad.rest.shape) * 1e-4
    xh = pad.rest + rng.normal(size=pad.rest.shape) * 1e-4
    p = rng.normal(size=x.shape)
    E, g, _ = En.inertia(x, xh, pad)
    j = En.inertia_line(x, p, xh, pad)
    assert float(j.v) == pytest.approx(E)
    assert float(j.d) == pytest.approx(float(np.sum(g * p)))
    assert float(j.dd) == pytest.approx(float(np.sum(pad.mass[:, None] * p * p)))


def test_taylor_arithmetic_against_closed_forms():
    t = T.Jet(np.array([0.7]), np.array([1.0]))        # the variable itself at 0.7
    f = T.log(t * t) / T.sqrt(t) + 3.0 * t
    v = 0.7
    # f = 2 ln v / sqrt(v) + 3 v
    f1 = 2 / v ** 1.5 - np.log(v) / v ** 1.5 + 3
    f2 = -3 / v ** 2.5 - (1 / v ** 2.5 - 1.5 * np.log(v) / v ** 2.5)
    assert float(f.v[0]) == pytest.approx(2 * np.log(v) / np.sqrt(v) + 3 * v)
    assert float(f.d[0]) == pytest.approx(f1)
    assert float(f.dd[0]) == pytest.approx(f2)
