"""Pins for the oracle RS-S factorization (CPU only).

What fixes each part, other than the oracle itself:
  * eps -> 0: with (numerically) full ranks RS-S is exact block Gaussian
    elimination, so the solve must reproduce the dense LU solve;
  * a single box (N <= s): the factorization is the dense LU of A;
  * solve/adjoint dot test <A^{-1} b, c> = <b, A^{-H} c> on the factored
    operator, and A^{-H} against the dense adjoint solve;
  * each ID against the explicit current far-field blocks A_FB and A_BF^T
    (brute force, Def. ID): ||A_FR - A_FS T|| <= 10 eps ||A_FB||;
  * ranks do not grow as eps is loosened (CPQR diagonal is non-increasing);
  * relative residual ||A x - b|| / ||b|| <= 10 eps (dense A);
  * CPQR against a brute-force greedy pivot order computed by least squares and
    the bound ||M_R - M_S T||_2 <= sqrt(r) eps ||M||_2.
Planted mistakes (a dropped Schur block, a transposed operand, a proxy sphere
that does not enclose the box) must fail them.
"""
import numpy as np
import pytest

import synth
from oracle import dense, kernel, rss
from oracle import tree as otree

K = 2.0 * np.pi


@pytest.fixture(scope="module")
def ell():
    s = synth.ellipsoid_uniform(2000, (1.0, 2.0, 0.5), seed=13)
    A = kernel.dense_matrix(s.points, s.normals, s.weights, K, K)
    b = synth.scaled_rhs(s, -synth.plane_wave(s.points, (0.0, 0.0, 1.0), K))
    xd = dense.solve(A, b)
    T = otree.build_tree(s.points, 24)
    return s, A, b, xd, T


def _factor(ell, eps, **kw):
    s, A, b, xd, T = ell
    rec = []
    F = rss.factor(s.points, s.normals, s.weights, K, eps, leaf_size=24, tree=T,
                   record=rec, snapshot_far=True, **kw)
    return F, rec


@pytest.fixture(scope="module")
def fac4(ell):
    return _factor(ell, 1e-4)


@pytest.fixture(scope="module")
def fac6(ell):
    return _factor(ell, 1e-6)


def _id_error_ratio(rec, eps):
    worst, count = 0.0, 0
    for r in rec:
        if r["R"].size == 0 or r["far"].size == 0:
            continue
        count += 1
        pos = {d: i for i, d in enumerate(r["act"])}
        si = [pos[d] for d in r["S"]]
        ri = [pos[d] for d in r["R"]]
        afb, abf = r["A_FB"], r["A_BF"]
        e1 = np.linalg.norm(afb[:, ri] - afb[:, si] @ r["T"], 2) / np.linalg.norm(afb, 2)
        e2 = np.linalg.norm(abf[ri, :].T - abf[si, :].T @ r["T"], 2) / np.linalg.norm(abf, 2)
        worst = max(worst, e1 / eps, e2 / eps)
    return worst, count


@pytest.mark.parametrize("which,eps", [("fac4", 1e-4), ("fac6", 1e-6)])
def test_residual_and_error_within_10eps(ell, which, eps, request):
    s, A, b, xd, T = ell
    F, rec = request.getfixturevalue(which)
    x = rss.solve(F, b)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 10 * eps
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 10 * eps
    assert len(F.boxes) > 20            # compression actually happened
    assert F.n0 < s.n


@pytest.mark.parametrize("which,eps", [("fac4", 1e-4), ("fac6", 1e-6)])
def test_id_against_dense_far_field(which, eps, request):
    F, rec = request.getfixturevalue(which)
    worst, count = _id_error_ratio(rec, eps)
    assert count > 20
    assert worst <= 10.0


def test_adjoint_dot_and_dense_adjoint(ell, fac4):
    s, A, b, xd, T = ell
    F, _ = fac4
    rng = np.random.default_rng(5)
    c = rng.standard_normal(s.n) + 1j * rng.standard_normal(s.n)
    lhs = np.vdot(c, rss.solve(F, b))
    rhs = np.vdot(rss.solve_adjoint(F, c), b)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    ya = rss.solve_adjoint(F, c)
    yd = dense.solve_adjoint(A, c)
    assert np.linalg.norm(ya - yd) / np.linalg.norm(yd) <= 1e-3


def test_eps_to_zero_reproduces_dense(ell):
    s, A, b, xd, T = ell
    F = rss.factor(s.points, s.normals, s.weights, K, 1e-14, leaf_size=24, tree=T)
    x = rss.solve(F, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-11


def test_single_box_is_dense_lu():
    s = synth.ellipsoid_uniform(50, (1.0, 2.0, 0.5), seed=3)
    A = kernel.dense_matrix(s.points, s.normals, s.weights, 3.0, 3.0)
    b = synth.scaled_rhs(s, synth.plane_wave(s.points, (1, 0, 0), 3.0))
    F = rss.factor(s.points, s.normals, s.weights, 3.0, 1e-6)
    assert len(F.boxes) == 0 and F.n0 == 50
    x = rss.solve(F, b)
    assert np.linalg.norm(x - dense.solve(A, b)) <= 1e-13 * np.linalg.norm(x)


def test_ranks_do_not_grow_as_eps_loosens(ell):
    s, A, b, xd, T = ell
    fin = T.nlevels - 1
    first, tot = {}, {}
    for eps in (1e-2, 1e-4, 1e-6, 1e-8):
        rec = []
        rss.factor(s.points, s.normals, s.weights, K, eps, leaf_size=24, tree=T,
                   record=rec)
        first[eps] = {r["box"]: r["S"].size for r in rec
                      if r["level"] == fin and r["colour"] == 0}
        tot[eps] = sum(r["S"].size for r in rec)
    epss = sorted(first)
    for lo, hi in zip(epss[:-1], epss[1:]):
        for B in first[lo]:
            assert first[hi][B] <= first[lo][B]
        assert tot[hi] <= tot[lo]


def _brute_greedy(M, steps):
    """Greedy pivots by least-squares residual norms (no QR updates)."""
    sel = []
    out = []
    for _ in range(steps):
        best, bi = -1.0, -1
        for j in range(M.shape[1]):
            if j in sel:
                continue
            if sel:
                coef = np.linalg.lstsq(M[:, sel], M[:, j], rcond=None)[0]
                res = np.linalg.norm(M[:, j] - M[:, sel] @ coef)
            else:
                res = np.linalg.norm(M[:, j])
            if res > best * (1 + 1e-12):
                best, bi = res, j
        sel.append(bi)
        out.append(best)
    return sel, np.array(out)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cpqr_against_brute_force(seed):
    rng = np.random.default_rng(seed)
    m, a, r = 60, 14, 7
    U = rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r))
    V = rng.standard_normal((r, a)) + 1j * rng.standard_normal((r, a))
    sv = np.logspace(0, -9, r)
    M = (U * sv) @ V + 1e-13 * (rng.standard_normal((m, a)))
    perm, rank, R = rss.cpqr(M, 1e-6)
    sel, res = _brute_greedy(M, rank)
    assert list(perm[:rank]) == sel
    assert np.allclose(np.abs(np.diag(R[:, :rank])), res, rtol=1e-6)
    d = np.abs(np.diag(R[:, :rank]))
    assert np.all(d[1:] <= d[:-1] * (1 + 1e-12))
    pv, s, T = rss.interp_decomp(M, 1e-6)
    assert s == rank
    err = np.linalg.norm(M[:, pv[s:]] - M[:, pv[:s]] @ T, 2)
    assert err <= np.sqrt(a - s) * 1e-6 * np.linalg.norm(M, 2)
    # the next pivot would fall below the threshold
    assert s == a or np.linalg.norm(M[:, pv[s:]] - M[:, pv[:s]] @ T, axis=0).max() \
        <= 1e-6 * d[0] * (1 + 1e-9)


# ---------------------------------------------------------------------------
# planted mistakes in the oracle must be caught by the pins above
# ---------------------------------------------------------------------------

def _residual_with(ell, monkeypatch, mutant, eps=1e-6):
    s, A, b, xd, T = ell
    monkeypatch.setattr(rss, "strong_skeletonize", mutant)
    F = rss.factor(s.points, s.normals, s.weights, K, eps, leaf_size=24, tree=T)
    x = rss.solve(F, b)
    return np.linalg.norm(A @ x - b) / np.linalg.norm(b)


def test_planted_dropped_schur_block_is_caught(ell, monkeypatch):
    def dropped(A, R, S, nd, T):
        ix = np.ix_
        keep = A[ix(nd, nd)].copy()
        out = good(A, R, S, nd, T)
        A[ix(nd, nd)] = keep            # forget the N x N Schur complement
        return out
    good = rss.strong_skeletonize
    assert _residual_with(ell, monkeypatch, dropped) > 10 * 1e-6   # the 10 eps pin fails


def test_planted_transposed_operand_is_caught(ell, monkeypatch):
    def transposed(A, R, S, nd, T):
        ix = np.ix_
        ASS = A[ix(S, S)].copy()
        A[ix(S, S)] = ASS.T             # A_SS^T where A_SS belongs
        out = good(A, R, S, nd, T)
        A[ix(S, S)] += ASS - ASS.T      # restore the original plus the update
        return out
    good = rss.strong_skeletonize
    assert _residual_with(ell, monkeypatch, transposed) > 10 * 1e-6


def test_planted_proxy_inside_box_is_caught(ell):
    # a proxy sphere of 0.5 x the half-diagonal leaves box points outside it,
    # so the proxy rows no longer span the far field (Sec. 5.1)
    F, rec = _factor(ell, 1e-4, proxy_factor=0.5)
    worst, _ = _id_error_ratio(rec, 1e-4)
    assert worst > 10.0


def test_proxy_sphere_near_the_far_boundary(ell):
    """Cross-check of the proxy radius reading: a sphere of 2.8 x the
    half-diagonal (2.42 h, just inside the 2.5 h ball that P never enters)
    gives IDs that still meet 10 eps against the explicit far field, a
    solution within 10 eps, and skeleton totals close to those of the
    default 1.5 x half-diagonal sphere."""
    s, A, b, xd, T = ell
    eps = 1e-4
    F, rec = _factor(ell, eps, proxy_factor=2.8)
    worst, count = _id_error_ratio(rec, eps)
    assert count > 20 and worst <= 10.0
    x = rss.solve(F, b)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 10 * eps
    F15, rec15 = _factor(ell, eps)
    s28 = sum(r["S"].size for r in rec)
    s15 = sum(r["S"].size for r in rec15)
    assert abs(s28 - s15) <= 0.15 * s15


def test_adaptive_proxy_count_rule():
    """The multipole estimate of the proxy count (Sec. 5.2): the floor for
    small boxes, growth with k rho, with the digits of accuracy, and the
    degree estimate p = ceil(k rho + 1.8 d^(2/3) (k rho)^(1/3)) at a value
    worked by hand: k rho = 8, eps = 1e-6 -> p = ceil(8 + 1.8 * 3.3019 * 2)
    = 20, 2 (p + 1)^2 = 882."""
    assert rss.proxy_count(1.0, 1e-3, 1e-6, 300) == 300
    assert rss.proxy_count(8.0, 1.0, 1e-6, 24) == 882
    counts = [rss.proxy_count(k, 0.5, 1e-6, 24) for k in (1.0, 4.0, 16.0, 64.0)]
    assert counts == sorted(counts) and counts[-1] > counts[0]
    assert rss.proxy_count(16.0, 0.5, 1e-10, 24) > rss.proxy_count(16.0, 0.5, 1e-3, 24)


def test_adaptive_proxy_ids_against_dense_far_field(ell):
    """With the per-level multipole count (floor 24 points) every ID still
    meets 10 eps against the explicit far field and the solution is within
    10 eps; the coarse levels use more points than the fine ones."""
    s, A, b, xd, T = ell
    eps = 1e-4
    F, rec = _factor(ell, eps, n_proxy=24, proxy_rule="adaptive")
    worst, count = _id_error_ratio(rec, eps)
    assert count > 20 and worst <= 10.0
    x = rss.solve(F, b)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 10 * eps
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 10 * eps
