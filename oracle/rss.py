"""Recursive strong skeletonization (RS-S) with proxy compression (oracle).

Test infrastructure: used only by tests, the smoke check and the benchmark's
CPU baseline. Plain and slow on purpose: the current matrix is kept dense and
every Schur complement is applied to it in place, so each step can be checked
by eye against the paper's formulas.

Steps, in the paper's order and notation:
  * Sec. 4.2 (RS-S): levels are processed from the finest to level 2; inside a
    level boxes go colour-major then Morton (the paper leaves the order free).
    A non-leaf box takes as actives the union of its children's skeletons.
    Processing stops early when no box of a level has active far DOFs.
  * Sec. 5.1 (simultaneous skeletonization): one ID of the stacked matrix
        [ A_QB ; A_BQ^T ; c K_{gamma B} sqrt(D_B) ; c S_{B gamma}^T sqrt(D_B) ]
    where A_QB holds the current entries (kernel plus Schur updates),
    K(y, x) = n(x).grad_x G(y, x) - i eta G(y, x) at proxy points y, and
    S_{B gamma}^T(l, j) = G(x_j, y_l). Proxy sphere: centre of B, radius
    1.5 x the half-diagonal of B, n_gamma Fibonacci points, rows scaled by
    c = sqrt(4 pi rho^2 / n_gamma) so that they are commensurate with the
    sqrt(w)-scaled rows (reading; the paper leaves the proxy rows unscaled).
  * Def. ID + greedy column-pivoted QR: Householder QR; at step j the pivot is
    the remaining column of largest norm, recomputed from the updated matrix,
    ties to the lowest index. Rank s = #{j : |R_jj| > eps |R_11|};
    T = R_11^{-1} R_12; S = first s pivots, R = the rest.
  * Eq. strong-skel-elim (Sec. 4.1): with T,
        X_RR = A_RR - T^T A_SR - A_RS T + T^T A_SS T
        X_RS = A_RS - T^T A_SS,   X_SR = A_SR - A_SS T
        X_RN = A_RN - T^T A_SN,   X_NR = A_NR - A_NS T
    (the R-F coupling is dropped), and the Schur complement
        A_{CC} -= X_{C R} X_RR^{-1} X_{R C},   C = S u N.
    Stored per box: T, X_RR^{-1}, X_{CR} = [X_SR; X_NR], X_{RC} = [X_RS X_RN].
  * Sec. 4.2 factored form: A^{-1} = W_1^{-1}..W_M^{-1} D^{-1} V_M^{-1}..V_1^{-1}
    with V^{-1} = L E P^T and W^{-1} = P F U. Forward sweep (elimination order)
        b_R -= T^T b_S ; z = X_RR^{-1} b_R ; b_C -= X_{CR} z ; b_R = z
    root solve with the dense LU of the remaining block, backward sweep
    (reverse order)
        x_R -= X_RR^{-1} X_{RC} x_C ; x_S -= T x_R .
    Adjoint (A^{-H} = V_1^{-H}..V_M^{-H} D^{-H} W_M^{-H}..W_1^{-H}): forward
        b_R -= T^H b_S ; z = X_RR^{-H} b_R ; b_C -= X_{RC}^H z ; b_R = z
    root A_tt^{-H}, backward
        x_R -= X_RR^{-H} X_{CR}^H x_C ; x_S -= conj(T) x_R .

Pins (tests/test_oracle_rss.py): eps -> 0 reproduces the dense solve; a single
box reduces to dense LU; the adjoint dot test; ranks do not grow as eps is
loosened; each ID checked against the explicit dense far-field block; residual
||Ax-b||/||b|| <= 10 eps; the CPQR against an SVD bound and a brute-force
pivot order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from . import kernel
from .tree import build_tree, current_boxes

GOLDEN_ANGLE = math.pi * (3.0 - math.sqrt(5.0))


def fibonacci_sphere(n: int) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * GOLDEN_ANGLE
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


# ---------------------------------------------------------------------------
# greedy column-pivoted QR and the interpolative decomposition (Def. ID)
# ---------------------------------------------------------------------------

def householder_vector(x: np.ndarray):
    """Reflector H = I - tau v v^H with H x = alpha e_1, |alpha| = ||x||."""
    nrm = np.linalg.norm(x)
    if nrm == 0.0:
        return np.zeros_like(x), 0.0, 0.0 + 0.0j
    x0 = x[0]
    phase = x0 / abs(x0) if x0 != 0 else 1.0
    alpha = -phase * nrm
    v = x.copy()
    v[0] -= alpha
    vv = np.vdot(v, v).real
    tau = 2.0 / vv if vv > 0 else 0.0
    return v, tau, alpha


def cpqr(M: np.ndarray, eps: float):
    """Greedy CPQR; returns (perm, rank, R) with R the s x a leading rows.

    Stops as soon as the pivot column norm is <= eps * |R_11|.
    """
    M = np.array(M, dtype=np.complex128, copy=True)
    m, a = M.shape
    perm = np.arange(a)
    rank = min(m, a)
    r11 = 0.0
    for j in range(min(m, a)):
        norms = np.sum(np.abs(M[j:, j:]) ** 2, axis=0)
        p = j + int(np.argmax(norms))
        if p != j:
            M[:, [j, p]] = M[:, [p, j]]
            perm[[j, p]] = perm[[p, j]]
        nrm = math.sqrt(norms[p - j])
        if j == 0:
            r11 = nrm
        if nrm <= eps * r11 or nrm == 0.0:
            rank = j
            break
        v, tau, alpha = householder_vector(M[j:, j])
        if j + 1 < a:
            w = v.conj() @ M[j:, j + 1:]
            M[j:, j + 1:] -= tau * np.outer(v, w)
        M[j, j] = alpha
        M[j + 1:, j] = 0.0
    return perm, rank, M[:rank, :]


def interp_decomp(M: np.ndarray, eps: float):
    """ID of the columns of M: M[:, R] ~ M[:, S] T. Returns (perm, s, T)."""
    perm, s, R = cpqr(M, eps)
    a = M.shape[1]
    if s == 0:
        return perm, 0, np.zeros((0, a), dtype=np.complex128)
    T = sla.solve_triangular(R[:, :s], R[:, s:], lower=False)
    return perm, s, T


# ---------------------------------------------------------------------------
# factorization
# ---------------------------------------------------------------------------

@dataclass
class BoxFactor:
    box: int
    level: int
    colour: int
    R: np.ndarray          # DOF ids (Morton-sorted numbering)
    S: np.ndarray
    N: np.ndarray
    T: np.ndarray          # s x r
    Xinv: np.ndarray       # r x r
    XCR: np.ndarray        # (s+n) x r  = [X_SR ; X_NR]
    XRC: np.ndarray        # r x (s+n)  = [X_RS , X_RN]


@dataclass
class Factorization:
    tree: object
    perm: np.ndarray
    k: float
    eta: float
    eps: float
    n: int
    boxes: list = field(default_factory=list)
    root_dofs: np.ndarray = None
    root_lu: tuple = None
    stop_level: int = 1
    ranks: dict = field(default_factory=dict)   # box -> (a, s, n_near, q)

    @property
    def n0(self) -> int:
        return int(self.root_dofs.size)


def proxy_count(k: float, rho: float, eps: float, n_min: int) -> int:
    """Frequency-adaptive number of proxy points (Sec. 5.2, proxy surface
    discretization: choose n_gamma from multipole estimates). Reading: the
    excess-bandwidth estimate of the truncation degree of a multipole
    expansion on a sphere of radius rho at accuracy eps,
        p = ceil(k rho + 1.8 d0^(2/3) (k rho)^(1/3)),  d0 = log10(1/eps),
    and twice the (p + 1)^2 spherical harmonics of degree <= p as sample
    points, never fewer than n_min."""
    kr = k * rho
    d0 = math.log10(1.0 / eps)
    p = math.ceil(kr + 1.8 * d0 ** (2.0 / 3.0) * kr ** (1.0 / 3.0))
    return max(int(n_min), 2 * (p + 1) ** 2)


def proxy_points(tree, box, n_proxy: int, proxy_factor: float, rule: str = "fixed",
                 k: float = 0.0, eps: float = 1.0):
    """Proxy sphere of `box`: centre of the box, radius proxy_factor x its
    half-diagonal, Fibonacci points. rule "fixed": n_proxy points; rule
    "adaptive": proxy_count(k, rho, eps, n_proxy) points."""
    b = tree.boxes[box]
    h = tree.side / float(1 << b.level)
    center = tree.corner + (np.array(b.cell, dtype=np.float64) + 0.5) * h
    rho = proxy_factor * (math.sqrt(3.0) / 2.0) * h
    if rule == "adaptive":
        n_proxy = proxy_count(k, rho, eps, n_proxy)
    elif rule != "fixed":
        raise ValueError(rule)
    return center[None, :] + rho * fibonacci_sphere(n_proxy), rho


def id_matrix(A, act_B, qd, x, nrm, sw, k, eta, Y, rho):
    """Stacked matrix of Sec. 5.1 (simultaneous skeletonization)."""
    nprox = Y.shape[0]
    cg = math.sqrt(4.0 * math.pi * rho * rho / nprox)
    a = act_B
    with np.errstate(divide="ignore", invalid="ignore"):
        kout = kernel.comb_kernel(Y, x[a], nrm[a], k, eta) * (cg * sw[a])[None, :]
        kin = kernel.green(x[a], Y, k).T * (cg * sw[a])[None, :]
    return np.vstack([A[np.ix_(qd, a)], A[np.ix_(a, qd)].T, kout, kin])


def strong_skeletonize(A, R, S, nd, T):
    """Eq. strong-skel-elim on the current dense matrix A (updated in place).

    Forms the X blocks, inverts X_RR (LU with partial pivoting) and applies the
    Schur complement to the (S u N) x (S u N) block. Returns the stored factors.
    """
    ix = np.ix_
    ARR, ARS = A[ix(R, R)], A[ix(R, S)]
    ASR, ASS = A[ix(S, R)], A[ix(S, S)]
    ARN, ANR = A[ix(R, nd)], A[ix(nd, R)]
    ASN, ANS = A[ix(S, nd)], A[ix(nd, S)]
    Tt = T.T
    XRR = ARR - Tt @ ASR - ARS @ T + Tt @ ASS @ T
    XRS = ARS - Tt @ ASS
    XSR = ASR - ASS @ T
    XRN = ARN - Tt @ ASN
    XNR = ANR - ANS @ T
    Xinv = sla.inv(XRR)
    XCR = np.vstack([XSR, XNR])
    XRC = np.hstack([XRS, XRN])
    C = np.concatenate([S, nd])
    A[ix(C, C)] -= XCR @ (Xinv @ XRC)
    return Xinv, XCR, XRC


def factor(points, normals, weights, k, eps, eta=None, leaf_size=64,
           n_proxy=300, proxy_factor=1.5, tree=None, record=None,
           snapshot_far=False, proxy_rule="fixed"):
    """RS-S factorization of the scaled CFIE system. Returns a Factorization.

    `record` (a list) receives one dict per processed box; with
    `snapshot_far` it also holds the current far-field blocks A_FB and A_BF
    (F = current actives outside B and N(B)) taken just before the ID.
    """
    eta = float(k) if eta is None else float(eta)
    points = np.asarray(points, dtype=np.float64)
    tr = build_tree(points, leaf_size) if tree is None else tree
    P = tr.perm
    x = points[P]
    nrm = np.asarray(normals, dtype=np.float64)[P]
    w = np.asarray(weights, dtype=np.float64)[P]
    sw = np.sqrt(w)
    A = kernel.dense_matrix(x, nrm, w, k, eta)        # current matrix
    F = Factorization(tree=tr, perm=P, k=float(k), eta=eta, eps=float(eps),
                      n=points.shape[0])
    act = {}
    for i, b in enumerate(tr.boxes):
        if b.leaf:
            act[i] = np.arange(b.start, b.end, dtype=np.int64)
    empty = np.zeros(0, dtype=np.int64)

    def merge(level):
        for i, b in enumerate(tr.boxes):
            if b.level == level and not b.leaf:
                act[i] = np.concatenate([act[c] for c in b.children])

    root_level = 1
    for lev in range(tr.nlevels - 1, 1, -1):
        L = tr.levels[lev]
        merge(lev)
        total = sum(act[C].size for C in L.current)
        far_any = False
        for B in L.boxes:
            closed = act[B].size + sum(act[C].size for C in L.near[B])
            if total - closed > 0:
                far_any = True
                break
        if not far_any:
            root_level = lev
            break
        for B in L.order:
            a = act[B]
            nd = np.concatenate([act[C] for C in L.near[B]] or [empty])
            qd = np.concatenate([act[C] for C in L.farq[B]] or [empty])
            Y, rho = proxy_points(tr, B, n_proxy, proxy_factor, proxy_rule, k, eps)
            M = id_matrix(A, a, qd, x, nrm, sw, k, eta, Y, rho)
            pv, s, T = interp_decomp(M, eps)
            S = a[pv[:s]]
            R = a[pv[s:]]
            F.ranks[B] = (int(a.size), int(s), int(nd.size), int(qd.size))
            if record is not None:
                item = dict(box=B, level=lev, colour=L.colour[B], act=a,
                            S=S, R=R, T=T, N=nd, Q=qd, perm=pv)
                if snapshot_far:
                    allact = np.concatenate([act[C] for C in L.current])
                    closed = np.concatenate([a, nd])
                    fd = np.setdiff1d(allact, closed)
                    item["far"] = fd
                    item["A_FB"] = A[np.ix_(fd, a)].copy()
                    item["A_BF"] = A[np.ix_(a, fd)].copy()
                record.append(item)
            act[B] = S
            if R.size == 0:
                continue
            Xinv, XCR, XRC = strong_skeletonize(A, R, S, nd, T)
            F.boxes.append(BoxFactor(B, lev, L.colour[B], R, S, nd, T, Xinv,
                                     XCR, XRC))
    if root_level == 1:
        merge(1)
    cur = current_boxes(tr, root_level)
    t = np.concatenate([act[C] for C in cur]) if cur else empty
    F.root_dofs = t
    F.stop_level = root_level
    F.root_lu = sla.lu_factor(A[np.ix_(t, t)]) if t.size else None
    return F


# ---------------------------------------------------------------------------
# factor application (Sec. 4.2) and its adjoint
# ---------------------------------------------------------------------------

def _to_sorted(F, b):
    b = np.asarray(b, dtype=np.complex128)
    return b[F.perm].copy()


def _from_sorted(F, bs):
    out = np.empty_like(bs)
    out[F.perm] = bs
    return out


def solve(F: Factorization, b: np.ndarray) -> np.ndarray:
    """x = A^{-1} b with the stored factors (b, x in the caller's point order)."""
    v = _to_sorted(F, b)
    for f in F.boxes:
        C = np.concatenate([f.S, f.N])
        bR = v[f.R] - f.T.T @ v[f.S]
        z = f.Xinv @ bR
        v[C] -= f.XCR @ z
        v[f.R] = z
    if F.root_lu is not None:
        v[F.root_dofs] = sla.lu_solve(F.root_lu, v[F.root_dofs])
    for f in reversed(F.boxes):
        C = np.concatenate([f.S, f.N])
        xR = v[f.R] - f.Xinv @ (f.XRC @ v[C])
        v[f.R] = xR
        v[f.S] -= f.T @ xR
    return _from_sorted(F, v)


def solve_adjoint(F: Factorization, b: np.ndarray) -> np.ndarray:
    """x = A^{-H} b with the stored factors."""
    v = _to_sorted(F, b)
    for f in F.boxes:
        C = np.concatenate([f.S, f.N])
        bR = v[f.R] - f.T.conj().T @ v[f.S]
        z = f.Xinv.conj().T @ bR
        v[C] -= f.XRC.conj().T @ z
        v[f.R] = z
    if F.root_lu is not None:
        v[F.root_dofs] = sla.lu_solve(F.root_lu, v[F.root_dofs], trans=2)
    for f in reversed(F.boxes):
        C = np.concatenate([f.S, f.N])
        xR = v[f.R] - f.Xinv.conj().T @ (f.XCR.conj().T @ v[C])
        v[f.R] = xR
        v[f.S] -= f.T.conj() @ xR
    return _from_sorted(F, v)


def factor_bytes(F: Factorization) -> int:
    """Complex128 bytes of the stored factors (m_f of Sec. 6)."""
    ent = 0
    for f in F.boxes:
        ent += f.T.size + f.Xinv.size + f.XCR.size + f.XRC.size
    ent += F.n0 * F.n0
    return 16 * ent
