"""Pins of the oracle's preconditioned GMRES (Sec. 7: a low-precision direct
solver used as a preconditioner) against what the mathematics fixes."""
import numpy as np
import pytest

import synth
from oracle import dense, gmres, kernel, rss


def _system(n=60, seed=3):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 2.0 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / (
        2.0 * np.sqrt(n))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    d = 1.0 / np.diag(A)                              # a rough (Jacobi) preconditioner
    return A, b, (lambda v: A @ v), (lambda v: d * v if v.ndim == 1 else d[:, None] * v)


@pytest.mark.parametrize("steps", [1, 2, 3, 5, 8])
def test_iterate_minimises_the_residual_over_the_krylov_space(steps):
    """After j steps (no restart) x_j = argmin ||b - A x|| over
    x in M^{-1} span{b, (A M^{-1}) b, ..., (A M^{-1})^{j-1} b}: brute force on
    an explicit (orthonormalised) Krylov basis gives the same residual."""
    A, b, fa, fm = _system()
    x, its, hist = gmres.gmres(fa, fm, b, tol=1e-300, restart=50, maxiter=steps)
    assert its == steps
    K = [b]
    for _ in range(steps - 1):
        K.append(fa(fm(K[-1])))
    Q, _ = np.linalg.qr(np.stack(K, axis=1))
    Z = fm(Q)
    y, *_ = np.linalg.lstsq(A @ Z, b, rcond=None)
    best = np.linalg.norm(b - A @ (Z @ y))
    got = np.linalg.norm(b - A @ x)
    assert abs(got - best) <= 1e-10 * np.linalg.norm(b)
    # the Givens estimate is the true residual of the iterate
    assert abs(hist[-1] - got / np.linalg.norm(b)) <= 1e-10


def test_exact_preconditioner_converges_in_one_step():
    A, b, fa, _ = _system(seed=5)
    x, its, hist = gmres.gmres(fa, lambda v: np.linalg.solve(A, v), b, tol=1e-12)
    assert its == 1
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)


def test_restarts_reach_the_tolerance():
    A, b, fa, fm = _system(seed=7)
    x, its, hist = gmres.gmres(fa, fm, b, tol=1e-12, restart=4, maxiter=200)
    assert np.linalg.norm(A @ x - b) <= 2e-12 * np.linalg.norm(b)
    assert its > 4                                     # more than one cycle was needed


def test_loose_rss_preconditioner_reaches_dense_accuracy():
    """A factorization at eps = 1e-2 preconditions GMRES on the dense CFIE
    matrix to 1e-12 in a few steps, and the result is the dense solve."""
    s = synth.ellipsoid_uniform(1500, (1.0, 2.0, 0.5), seed=13)
    k = 2.0 * np.pi
    A = kernel.dense_matrix(s.points, s.normals, s.weights, k, k)
    b = synth.scaled_rhs(s, -synth.plane_wave(s.points, (0.0, 0.0, 1.0), k))
    F = rss.factor(s.points, s.normals, s.weights, k, 1e-2, leaf_size=24)
    x, its, hist = gmres.gmres(lambda v: A @ v, lambda v: rss.solve(F, v), b, tol=1e-12)
    assert its <= 8
    xd = dense.solve(A, b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert all(h2 <= h1 * (1 + 1e-12) for h1, h2 in zip(hist, hist[1:]))   # monotone


def test_planted_wrong_rotation_is_caught(monkeypatch):
    """A rotation with the wrong conjugation breaks the minimal-residual pin."""
    good = gmres.givens

    def bad(f, g):
        c, s, r = good(f, g)
        return c, np.conj(s), r

    monkeypatch.setattr(gmres, "givens", bad)
    A, b, fa, fm = _system()
    x, its, hist = gmres.gmres(fa, fm, b, tol=1e-300, restart=50, maxiter=5)
    got = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert abs(hist[-1] - got) > 1e-6
