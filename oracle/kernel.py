"""Helmholtz combined-field kernel and the dense sqrt(w)-scaled system matrix.

Test infrastructure (oracle): used only by tests, the smoke check and the
benchmark's CPU baseline.

Definitions followed (Sec. 3):
  G(x, y) = exp(i k |x-y|) / (4 pi |x-y|)                       (Eq. greenfunhelm)
  K(x, y) = n(y) . grad_y G(x, y) - i eta G(x, y),  eta = k      (Eq. comb_ref)
  A_ij = sqrt(w_i) K(x_i, x_j) sqrt(w_j),  i != j               (Eq. disc3)
  A_ii = 1/2 + 0 - i eta (sqrt(w_i/pi)/2 + i k w_i/(4 pi))

The diagonal keeps the jump 1/2 of the exterior double layer, sets the
double-layer self term to 0 and replaces the single-layer self term by the
two-term expansion of the integral of G over a disc of area w_i centred at x_i,
(exp(i k a) - 1)/(2 i k) with a = sqrt(w_i/pi).

With r = x - y and d = |r|: grad_y G = G (i k d - 1)/d^2 (y - x).

Pins: tests/test_oracle_kernel.py checks the double-layer gradient against
finite differences of G, the Helmholtz equation for G, the self term against
numerical quadrature of G over the disc, the eigenvalues of the CFIE on the unit
sphere (closed form from the addition theorem) and the analytic point-source
test of Sec. 6.1.
"""
from __future__ import annotations

import math

import numpy as np

FOUR_PI = 4.0 * math.pi


def green(x: np.ndarray, y: np.ndarray, k: float) -> np.ndarray:
    """G(x_i, y_j) for targets x (m,3), sources y (n,3) -> (m, n)."""
    d = np.linalg.norm(x[:, None, :] - y[None, :, :], axis=2)
    return np.exp(1j * k * d) / (FOUR_PI * d)


def dlp_kernel(x: np.ndarray, y: np.ndarray, ny: np.ndarray, k: float) -> np.ndarray:
    """n(y_j) . grad_y G(x_i, y_j) -> (m, n)."""
    diff = y[None, :, :] - x[:, None, :]               # y - x
    d = np.linalg.norm(diff, axis=2)
    g = np.exp(1j * k * d) / (FOUR_PI * d)
    proj = np.einsum("mnc,nc->mn", diff, ny)            # (y - x) . n(y)
    return g * (1j * k * d - 1.0) / (d * d) * proj


def comb_kernel(x: np.ndarray, y: np.ndarray, ny: np.ndarray, k: float,
                eta: float) -> np.ndarray:
    """K(x_i, y_j) = n(y_j).grad_y G - i eta G -> (m, n)."""
    return dlp_kernel(x, y, ny, k) - 1j * eta * green(x, y, k)


def self_term(w: np.ndarray, k: float, eta: float) -> np.ndarray:
    """Diagonal A_ii = 1/2 - i eta (sqrt(w/pi)/2 + i k w/(4 pi))."""
    s_self = np.sqrt(w / math.pi) / 2.0 + 1j * k * w / FOUR_PI
    return 0.5 - 1j * eta * s_self


def matrix_block(rows: np.ndarray, cols: np.ndarray, x: np.ndarray,
                 nrm: np.ndarray, w: np.ndarray, k: float, eta: float) -> np.ndarray:
    """Entries A[rows, cols] of the scaled system (no Schur updates)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    if rows.size == 0 or cols.size == 0:
        return np.zeros((rows.size, cols.size), dtype=np.complex128)
    same = rows[:, None] == cols[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        kk = comb_kernel(x[rows], x[cols], nrm[cols], k, eta)
    blk = np.sqrt(w[rows])[:, None] * kk * np.sqrt(w[cols])[None, :]
    if same.any():
        ii, jj = np.nonzero(same)
        blk[ii, jj] = self_term(w[rows[ii]], k, eta)
    return blk


def dense_matrix(x: np.ndarray, nrm: np.ndarray, w: np.ndarray, k: float,
                 eta: float | None = None) -> np.ndarray:
    """The full N x N scaled system matrix A (Eq. disc3 with the disc self term)."""
    eta = k if eta is None else eta
    n = x.shape[0]
    idx = np.arange(n)
    out = np.empty((n, n), dtype=np.complex128)
    step = 1024
    for i0 in range(0, n, step):
        out[i0:i0 + step] = matrix_block(idx[i0:i0 + step], idx, x, nrm, w, k, eta)
    return out


def matvec(x: np.ndarray, nrm: np.ndarray, w: np.ndarray, k: float, eta: float,
           v: np.ndarray, rows: np.ndarray | None = None) -> np.ndarray:
    """(A v)[rows] without forming A; v is (N,) or (N, nrhs)."""
    n = x.shape[0]
    rows = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    idx = np.arange(n)
    vv = v if v.ndim == 2 else v[:, None]
    out = np.empty((rows.size, vv.shape[1]), dtype=np.complex128)
    step = max(1, 4_000_000 // max(n, 1))
    for i0 in range(0, rows.size, step):
        r = rows[i0:i0 + step]
        out[i0:i0 + step] = matrix_block(r, idx, x, nrm, w, k, eta) @ vv
    return out if v.ndim == 2 else out[:, 0]


def potential(targets: np.ndarray, x: np.ndarray, nrm: np.ndarray, w: np.ndarray,
              k: float, eta: float, sigma_tilde: np.ndarray) -> np.ndarray:
    """u(t) = sum_j K(t, x_j) sqrt(w_j) sigma~_j (combined-field layer potential)."""
    kk = comb_kernel(targets, x, nrm, k, eta)
    return kk @ (np.sqrt(w)[:, None] * sigma_tilde if sigma_tilde.ndim == 2
                 else np.sqrt(w) * sigma_tilde)
