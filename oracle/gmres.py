"""GMRES preconditioned by a loose RS-S factorization (oracle).

Test infrastructure: used only by the tests and the benchmark's CPU baseline.

The paper's conclusions (Sec. 7) note that the direct solver can instead be
run at low precision and used as a preconditioner for an iterative method.
This is that combination, written plainly: restarted GMRES with right
preconditioning,
    A M^{-1} u = b,   x = M^{-1} u,
where M^{-1} applies the stored factors of a factorization at a loose
tolerance (rss.solve) and A is the dense system matrix (or any product).
Each cycle builds an orthonormal Krylov basis V of A M^{-1} by classical
Gram-Schmidt applied twice, reduces the Hessenberg matrix H to triangular
form with Givens rotations as the basis grows (so |g_{j+1}| is the residual
norm of the least-squares problem min_y ||beta e_1 - H y||), and stops when
that estimate falls below tol ||b||; the update is x += M^{-1} (V y).

Pins (tests/test_oracle_gmres.py): the iterate after j steps minimises the
residual over the Krylov space (checked against a brute-force least-squares
solve on an explicit Krylov basis); an exact preconditioner converges in one
step; the converged x equals the dense solve; the estimate equals the true
residual.
"""
from __future__ import annotations

import numpy as np


def givens(f: complex, g: complex):
    """(c, s, r) with [c s; -conj(s) c] [f; g] = [r; 0], c real >= 0."""
    if g == 0:
        return 1.0, 0.0 + 0.0j, f
    if f == 0:
        return 0.0, np.conj(g) / abs(g), abs(g)
    af = abs(f)
    nrm = np.hypot(af, abs(g))
    c = af / nrm
    s = (f / af) * np.conj(g) / nrm
    r = (f / af) * nrm
    return c, s, r


def gmres(apply_a, apply_minv, b: np.ndarray, tol: float = 1e-10, restart: int = 30,
          maxiter: int = 200):
    """Solve A x = b. Returns (x, iterations, history of residual estimates
    relative to ||b||, one per step)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    hist = []
    if bnorm == 0.0:
        return x, 0, hist
    its = 0
    while its < maxiter:
        r = b - apply_a(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            break
        m = min(restart, maxiter - its)
        V = np.zeros((n, m + 1), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[:, 0] = r / beta
        j_done = 0
        for j in range(m):
            w = apply_a(apply_minv(V[:, j]))
            # classical Gram-Schmidt, twice
            h = V[:, :j + 1].conj().T @ w
            w = w - V[:, :j + 1] @ h
            h2 = V[:, :j + 1].conj().T @ w
            w = w - V[:, :j + 1] @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0:
                V[:, j + 1] = w / hn
            # earlier rotations on the new column, then a new one
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            c, s, rr = givens(H[j, j], H[j + 1, j])
            cs[j], sn[j] = c, s
            H[j, j] = rr
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            its += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or hn == 0:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + apply_minv(V[:, :j_done] @ y)
        if hist and hist[-1] <= tol:
            break
    return x, its, hist
