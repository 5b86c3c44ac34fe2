"""Pins of the CMA-ES driver (host logic, no device work).

On test functions whose minimiser is known: the sphere (minimiser inside
the cube and at a corner, reached through the reflection at the faces) and
a rotated ill-conditioned ellipsoid. A method that adapted only its step
size would need orders of magnitude more generations there; CMA-ES learns
the covariance. Also checked: the strategy uses only the ranking of the
objective values (identical runs under a strictly increasing transform of
f), and its default weights and learning rates obey the published
constraints (weights positive, decreasing and summing to 1; c1 + cmu <= 1).
"""
import numpy as np

from paper_2603_28475_b300 import calibrate as C


def _run(f, x0, sigma0, gens, seed=0, n=4):
    es = C.CMAES(x0, sigma0, popsize=12, seed=seed)
    for _ in range(gens):
        X = es.ask()
        assert np.all((X >= 0) & (X <= 1))
        es.tell([f(x) for x in X])
    return es


def test_sphere_inside_the_cube():
    opt = np.array([0.3, 0.62, 0.5, 0.71])
    es = _run(lambda x: float(np.sum((x - opt) ** 2)), np.full(4, 0.5), 0.3, 150)
    assert es.best_f < 1e-12
    assert np.abs(es.m - opt).max() < 1e-5


def test_sphere_minimiser_at_a_corner():
    opt = np.array([0.0, 1.0, 0.0, 1.0])
    es = _run(lambda x: float(np.sum((x - opt) ** 2)), np.full(4, 0.5), 0.3, 200)
    assert es.best_f < 1e-10


def test_rotated_ellipsoid_is_learned():
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    H = Q @ np.diag([1.0, 1e2, 1e4, 1e6]) @ Q.T
    opt = np.array([0.4, 0.45, 0.55, 0.6])
    f = lambda x: float((x - opt) @ H @ (x - opt))
    es = _run(f, np.full(4, 0.5), 0.2, 400)
    assert es.best_f < 1e-10
    # the learned covariance is aligned with H^-1: C H is close to a multiple of I
    CH = es.C @ H
    ev = np.linalg.eigvals(CH).real
    assert ev.max() / ev.min() < 1e3           # against a condition of 1e6 for C = I


def test_only_the_ranking_matters():
    opt = np.array([0.2, 0.8, 0.35, 0.5])
    f = lambda x: float(np.sum((x - opt) ** 2))
    a = _run(f, np.full(4, 0.5), 0.3, 30, seed=3)
    b = _run(lambda x: np.exp(f(x)) * 7.0 + 3.0, np.full(4, 0.5), 0.3, 30, seed=3)
    assert np.array_equal(a.m, b.m) and a.sigma == b.sigma and np.array_equal(a.C, b.C)


def test_strategy_parameters_obey_the_published_constraints():
    es = C.CMAES(np.full(4, 0.5), 0.3, popsize=12)
    assert es.mu == 6 and np.all(es.w > 0) and np.all(np.diff(es.w) < 0)
    assert abs(es.w.sum() - 1.0) < 1e-15
    assert 1.0 < es.mueff < es.mu
    assert 0 < es.c1 and 0 < es.cmu and es.c1 + es.cmu <= 1.0
    assert 0 < es.cs < 1 and 0 < es.cc <= 1 and es.ds > 1


def test_reflection_and_parameter_maps():
    x = np.array([-0.25, 1.25, 2.5, 0.5, -1.75])
    assert np.allclose(C.reflect_unit(x), [0.25, 0.75, 0.5, 0.5, 0.25])
    th = C.to_theta([0.0, 1.0, 0.5, 0.25])
    assert np.allclose(th, [1e4, 0.497, 3e3, 0.25 + 0.25 * 2.25])
    assert np.allclose(C.to_unit(th), [0.0, 1.0, 0.5, 0.25])
