"""Monostatic sonar cross section (oracle, Sec. 6.3).

Test infrastructure: used only by the tests and the benchmark's CPU baseline.

Incident plane wave u_inc = exp(i k d.x) travelling along the unit vector d;
sound-soft data f = -u_inc, so the scaled right-hand side is
b_j = -sqrt(w_j) exp(i k d.x_j). The scattered field is the combined-field
layer potential u(t) = sum_j K(t, x_j) sqrt(w_j) x~_j of the solution
x~ = sqrt(w) sigma. Its far-field pattern (u = e^{ikr}/r F + O(1/r^2)) in the
direction t^ follows from the large-|t| form of K,
    F(t^) = (1/(4 pi)) sum_j sqrt(w_j) x~_j exp(-i k t^.x_j) (-i k n_j.t^ - i eta),
and the monostatic cross section is its value back toward the source,
t^ = -d:
    R(d) = (1/(4 pi)) sum_j sqrt(w_j) x~_j exp(i k d.x_j) (i k n_j.d - i eta)
         = (-i k/(4 pi)) sum_j sqrt(w_j) x~_j exp(i k d.x_j) (1 - n_j.d),  eta = k.
Reading: the paper prints the exponential as exp(-i k x.d) next to the
factor (1 - n.d); the backscatter direction -d gives exp(+i k x.d), and the
pin in tests/test_oracle_sonar.py (the far-field limit of the potential
itself) confirms that sign.
"""
from __future__ import annotations

import math

import numpy as np


def azimuthal_directions(phis) -> np.ndarray:
    """Unit directions (cos phi, sin phi, 0) of an azimuthal sweep."""
    ph = np.asarray(phis, dtype=np.float64)
    return np.stack([np.cos(ph), np.sin(ph), np.zeros_like(ph)], axis=1)


def plane_wave_rhs(points: np.ndarray, weights: np.ndarray, k: float,
                   dirs: np.ndarray) -> np.ndarray:
    """b[:, m] = -sqrt(w) exp(i k d_m . x)  -> (N, M)."""
    return -np.sqrt(weights)[:, None] * np.exp(1j * k * (points @ dirs.T))


def far_field(points, normals, weights, k, eta, sol, that) -> np.ndarray:
    """F(t^_m) for the columns sol[:, m] and directions that[m] -> (M,)."""
    ph = np.exp(-1j * k * (points @ that.T))                       # (N, M)
    fac = -1j * k * (normals @ that.T) - 1j * eta                  # (N, M)
    return np.sum(np.sqrt(weights)[:, None] * sol * ph * fac, axis=0) / (4.0 * math.pi)


def backscatter(points, normals, weights, k, eta, dirs, sol) -> np.ndarray:
    """R(d_m) = F(-d_m) of solution column m (the wave along d_m)."""
    return far_field(points, normals, weights, k, eta, sol, -np.asarray(dirs))
