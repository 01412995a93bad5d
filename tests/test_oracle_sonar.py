"""Pins of the oracle's sonar cross section (Sec. 6.3): the far-field formula
against the potential itself far away, and the monostatic backscatter of a
sound-soft sphere against its closed-form (Mie) series."""
import math

import numpy as np
import pytest
from scipy import special

import synth
from oracle import dense, kernel, sonar


def test_far_field_is_the_limit_of_the_potential():
    """r e^{-ikr} u(r t^) -> F(t^) with an O(1/r) error."""
    s = synth.ellipsoid_uniform(400, (1.0, 2.0, 0.5), seed=4)
    k, eta = 3.0, 3.0
    rng = np.random.default_rng(1)
    sol = (rng.standard_normal((s.n, 3)) + 1j * rng.standard_normal((s.n, 3)))
    that = synth.seeded_directions(3, 9)
    F = sonar.far_field(s.points, s.normals, s.weights, k, eta, sol, that)
    errs = []
    for r in (1e3, 1e4, 1e5):
        u = np.array([kernel.potential((r * that[m])[None, :], s.points, s.normals, s.weights,
                                       k, eta, sol[:, m])[0] for m in range(3)])
        errs.append(np.max(np.abs(u * r * np.exp(-1j * k * r) - F) / np.abs(F)))
    assert errs[2] < 1e-3
    assert errs[2] < 0.2 * errs[1] < 0.04 * errs[0]


def _mie_backscatter(k, a=1.0, terms=60):
    n = np.arange(terms)
    jn = special.spherical_jn(n, k * a)
    hn = jn + 1j * special.spherical_yn(n, k * a)
    return (1j / k) * np.sum((2 * n + 1) * (-1.0) ** n * jn / hn)


def _sphere_backscatter(n, k, phis):
    s = synth.sphere_fibonacci(n)
    dirs = sonar.azimuthal_directions(phis)
    A = kernel.dense_matrix(s.points, s.normals, s.weights, k, k)
    B = sonar.plane_wave_rhs(s.points, s.weights, k, dirs)
    X = dense.solve(A, B)
    return sonar.backscatter(s.points, s.normals, s.weights, k, k, dirs, X)


def test_sound_soft_sphere_backscatter_matches_mie_series():
    """The monostatic cross section of the unit sphere (all azimuths equal by
    symmetry) converges at first order in h to the Mie series; the forward
    value (the other sign of the exponential) is far from it."""
    k = 2.0
    exact = _mie_backscatter(k)
    phis = np.linspace(0.0, 2.0 * math.pi, 5, endpoint=False)
    e = []
    for n in (1000, 4000):
        R = _sphere_backscatter(n, k, phis)
        e.append(np.max(np.abs(R - exact)) / abs(exact))
    assert e[1] < 0.03
    assert e[1] < 0.7 * e[0]
    nn = np.arange(60)
    jn = special.spherical_jn(nn, k)
    hn = jn + 1j * special.spherical_yn(nn, k)
    forward = (1j / k) * np.sum((2 * nn + 1) * jn / hn)
    assert abs(forward - exact) > 10 * e[1] * abs(exact)


def test_planted_wrong_exponent_sign_is_caught(monkeypatch):
    """Using exp(-i k d.x) (the forward direction) fails the Mie pin."""
    monkeypatch.setattr(sonar, "backscatter",
                        lambda p, nr, w, k, eta, dirs, sol: sonar.far_field(p, nr, w, k, eta, sol,
                                                                            np.asarray(dirs)))
    k = 2.0
    R = _sphere_backscatter(2000, k, [0.3])
    exact = _mie_backscatter(k)
    assert abs(R[0] - exact) / abs(exact) > 0.1
