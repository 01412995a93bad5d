"""Pins for the oracle's kernel and dense system matrix (CPU only).

Each check compares the oracle with something other than itself:
  * finite differences of G (the double-layer gradient, the Helmholtz equation);
  * 2-D numerical quadrature of G over a disc (the single-layer self term);
  * the closed-form CFIE eigenvalues on the unit sphere (addition theorem:
    lambda_n = i k^2 j_n'(k) h_n(k) + eta k j_n(k) h_n(k), scipy.special);
  * the analytic test of Sec. 6.1: Dirichlet data from an interior point
    source must reproduce its field at exterior targets (uniqueness of the
    exterior Dirichlet problem, Eq. extdir).
Planted mistakes (a flipped double-layer sign, the target normal in place of
the source normal, a dropped self term) are shown to fail these pins.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import spherical_jn, spherical_yn

import synth
from oracle import dense, kernel


def _lam(n, k, eta):
    j = spherical_jn(n, k)
    jp = spherical_jn(n, k, derivative=True)
    h = j + 1j * spherical_yn(n, k)
    return 1j * k * k * jp * h + eta * k * j * h


def test_green_solves_helmholtz():
    k = 2.3
    y = np.array([[0.1, -0.2, 0.3]])
    x0 = np.array([0.9, 0.4, -0.5])
    h = 1e-3
    lap = -6.0 * kernel.green(x0[None, :], y, k)[0, 0]
    for c in range(3):
        for s in (1, -1):
            xp = x0.copy()
            xp[c] += s * h
            lap += kernel.green(xp[None, :], y, k)[0, 0]
    lap /= h * h
    g0 = kernel.green(x0[None, :], y, k)[0, 0]
    assert abs(lap + k * k * g0) < 1e-4 * abs(k * k * g0)


def test_double_layer_is_source_normal_derivative():
    rng = np.random.default_rng(3)
    k = 1.7
    x = rng.standard_normal((4, 3))
    y = rng.standard_normal((5, 3)) + 3.0
    ny = rng.standard_normal((5, 3))
    ny /= np.linalg.norm(ny, axis=1, keepdims=True)
    d = kernel.dlp_kernel(x, y, ny, k)
    h = 1e-5
    fd = (kernel.green(x, y + h * ny, k) - kernel.green(x, y - h * ny, k)) / (2 * h)
    # column j of fd uses y_j moved along n_j: compare entrywise per column
    fd_cols = np.empty_like(d)
    for j in range(y.shape[0]):
        yp = y[j:j + 1] + h * ny[j:j + 1]
        ym = y[j:j + 1] - h * ny[j:j + 1]
        fd_cols[:, j] = ((kernel.green(x, yp, k) - kernel.green(x, ym, k)) / (2 * h))[:, 0]
    assert np.allclose(d, fd_cols, rtol=1e-7, atol=1e-9)
    assert fd.shape == d.shape


@pytest.mark.parametrize("w,k,eta", [(4 * math.pi / 2000, 1.0, 1.0),
                                     (1e-3, 6.0, 6.0), (2e-4, 20.0, 20.0)])
def test_self_term_matches_disc_quadrature(w, k, eta):
    a = math.sqrt(w / math.pi)

    def integrand(r, th, part):
        x = np.array([[0.0, 0.0, 0.0]])
        y = np.array([[r * math.cos(th), r * math.sin(th), 0.0]])
        g = kernel.green(x, y, k)[0, 0] * r
        return g.real if part == 0 else g.imag

    re = integrate.dblquad(lambda r, th: integrand(r, th, 0), 0, 2 * math.pi, 1e-14, a,
                           epsabs=1e-13)[0]
    im = integrate.dblquad(lambda r, th: integrand(r, th, 1), 0, 2 * math.pi, 1e-14, a,
                           epsabs=1e-13)[0]
    s_disc = re + 1j * im
    diag = kernel.self_term(np.array([w]), k, eta)[0]
    s_oracle = (diag - 0.5) / (-1j * eta)
    # two-term expansion: error of the next term, k^2 a^3 / 12
    assert abs(s_oracle - s_disc) <= 0.2 * k * k * a ** 3 + 1e-12


def test_closed_form_eigenvalues_match_golden():
    """The spherical-Bessel closed form used below agrees with the golden
    values written out in elementary functions (tests/golden, two degrees,
    two wavenumbers)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "sphere_cfie_eigenvalues.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 4
    for n, k, eta, re_, im_ in rows:
        want = complex(float(re_), float(im_))
        assert abs(_lam(int(n), float(k), float(eta)) - want) <= 1e-12 * abs(want)


@pytest.mark.parametrize("n_harm", [0, 1, 2])
def test_sphere_eigenvalues_converge(n_harm):
    k = eta = 1.0
    lam = _lam(n_harm, k, eta)
    errs = []
    for n in (1000, 4000):
        s = synth.sphere_fibonacci(n)
        A = kernel.dense_matrix(s.points, s.normals, s.weights, k, eta)
        z = s.points[:, 2]
        Y = [np.ones(n), z, (3 * z * z - 1) / 2][n_harm]
        v = np.sqrt(s.weights) * Y
        rq = np.vdot(v, A @ v) / np.vdot(v, v)
        errs.append(abs(rq - lam))
    assert errs[0] < 0.02
    assert errs[1] < 0.0095
    assert errs[0] / errs[1] > 1.8            # first order in h ~ N^{-1/2}


def _analytic_error(surface, k, src):
    A = kernel.dense_matrix(surface.points, surface.normals, surface.weights, k, k)
    b = synth.scaled_rhs(surface, synth.point_source_field(surface.points, src, k))
    x = dense.solve(A, b)
    t = synth.exterior_targets(50, 3.0)
    u = kernel.potential(t, surface.points, surface.normals, surface.weights, k, k, x)
    ue = synth.point_source_field(t, src, k)
    return np.linalg.norm(u - ue) / np.linalg.norm(ue), A, x, b


def test_analytic_point_source_sphere():
    e1, A, x, b = _analytic_error(synth.sphere_fibonacci(1000), 1.0, (0.1, 0.2, -0.1))
    e2, *_ = _analytic_error(synth.sphere_fibonacci(4000), 1.0, (0.1, 0.2, -0.1))
    assert e1 < 0.03 and e2 < 0.015
    assert e1 / e2 > 1.6
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-12


def test_analytic_accuracy_metric_as_printed():
    """The accuracy measure of Sec. 6.1 divides the target-error norm by
    the L2 norm of the density on the surface, sqrt(int |sigma|^2 da), which
    the scaled unknowns give as ||x||_2 (x = sqrt(w) sigma). Both that
    measure and the plain relative error fall at first order in h."""
    out = []
    for n in (1000, 4000):
        s = synth.sphere_fibonacci(n)
        e_rel, A, x, b = _analytic_error(s, 1.0, (0.1, 0.2, -0.1))
        t = synth.exterior_targets(50, 3.0)
        u = kernel.potential(t, s.points, s.normals, s.weights, 1.0, 1.0, x)
        ue = synth.point_source_field(t, (0.1, 0.2, -0.1), 1.0)
        e_a = np.linalg.norm(u - ue) / np.linalg.norm(x)
        out.append((e_rel, e_a))
    (r1, a1), (r2, a2) = out
    assert a1 < 0.02 and a2 < 0.01
    assert a1 / a2 > 1.6 and r1 / r2 > 1.6


def test_analytic_point_source_ellipsoid():
    s = synth.ellipsoid_uniform(3000, (1.0, 2.0, 0.5), seed=11)
    e, *_ = _analytic_error(s, 2.0, (0.2, 0.5, 0.05))
    assert e < 0.05


# ---------------------------------------------------------------------------
# planted mistakes: each must break a pin above
# ---------------------------------------------------------------------------

def test_planted_sign_flip_is_caught(monkeypatch):
    good = kernel.dlp_kernel
    monkeypatch.setattr(kernel, "dlp_kernel", lambda *a: -good(*a))
    s = synth.sphere_fibonacci(1000)
    A = kernel.dense_matrix(s.points, s.normals, s.weights, 1.0, 1.0)
    v = np.sqrt(s.weights)
    rq = np.vdot(v, A @ v) / np.vdot(v, v)
    assert abs(rq - _lam(0, 1.0, 1.0)) > 0.1


def test_planted_target_normal_is_caught(monkeypatch):
    def wrong(x, y, ny, k):
        # uses the normal at the target instead of the source
        diff = y[None, :, :] - x[:, None, :]
        d = np.linalg.norm(diff, axis=2)
        g = np.exp(1j * k * d) / (4 * np.pi * d)
        nx = x / np.linalg.norm(x, axis=1, keepdims=True) * np.array([1.0, 0.25, 4.0])
        nx /= np.linalg.norm(nx, axis=1, keepdims=True)
        proj = -np.einsum("mnc,mc->mn", diff, nx)
        return g * (1j * k * d - 1.0) / (d * d) * proj
    monkeypatch.setattr(kernel, "dlp_kernel", wrong)
    s = synth.ellipsoid_uniform(3000, (1.0, 2.0, 0.5), seed=11)
    e, *_ = _analytic_error(s, 2.0, (0.2, 0.5, 0.05))
    assert e > 0.1


def test_planted_missing_self_term_is_caught(monkeypatch):
    monkeypatch.setattr(kernel, "self_term", lambda w, k, eta: 0.5 + 0.0 * w)
    s = synth.sphere_fibonacci(1000)
    A = kernel.dense_matrix(s.points, s.normals, s.weights, 1.0, 1.0)
    v = np.sqrt(s.weights)
    rq = np.vdot(v, A @ v) / np.vdot(v, v)
    assert abs(rq - _lam(0, 1.0, 1.0)) > 0.02
