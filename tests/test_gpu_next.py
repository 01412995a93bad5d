"""GPU parity of the extensions beyond the direct solve, against the oracle:
  * frequency-adaptive proxy counts per level (Sec. 5.2);
  * GMRES preconditioned by a loose factorization (Sec. 7);
  * the monostatic sonar cross section over an azimuthal sweep (Sec. 6.3).
"""
import math

import numpy as np
import pytest

import synth
from oracle import dense, gmres as ogmres, kernel, rss, sonar

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 2.0 * np.pi


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_07325_gb300 as p
    p.load_library()
    return p


@pytest.fixture(scope="module")
def ell():
    s = synth.ellipsoid_uniform(2000, (1.0, 2.0, 0.5), seed=13)
    A = kernel.dense_matrix(s.points, s.normals, s.weights, K, K)
    b = synth.scaled_rhs(s, -synth.plane_wave(s.points, (0.0, 0.0, 1.0), K))
    return s, A, b, dense.solve(A, b)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------------------
# adaptive proxy counts
# ---------------------------------------------------------------------------

def test_adaptive_proxy_counts_match_oracle(pkg, ell):
    s, A, b, xd = ell
    eps, floor = 1e-4, 24
    fac = pkg.Factorization(s.points, s.normals, s.weights, K, eps, leaf_size=24,
                            precision=pkg.PRECISION_FP64, n_proxy=floor,
                            proxy_rule=pkg.PROXY_ADAPTIVE)
    try:
        st = fac.stats()
        x = fac.solve(torch.from_numpy(b)).cpu().numpy()
    finally:
        fac.free()
    F = rss.factor(s.points, s.normals, s.weights, K, eps, leaf_size=24, n_proxy=floor,
                   proxy_rule="adaptive")
    xo = rss.solve(F, b)
    T = F.tree
    for lv in st["levels"]:
        h = T.side / 2 ** lv["level"]
        rho = 1.5 * (math.sqrt(3.0) / 2.0) * h
        assert lv["n_proxy"] == rss.proxy_count(K, rho, eps, floor), lv
        L = T.levels[lv["level"]]
        sum_s = sum(F.ranks[B][1] for B in L.boxes if B in F.ranks)
        assert abs(lv["sum_s"] - sum_s) <= max(2, 0.01 * sum_s), lv
    # the coarse levels get more than the floor, the count grows with the box
    counts = [lv["n_proxy"] for lv in sorted(st["levels"], key=lambda l: l["level"])]
    assert counts == sorted(counts, reverse=True) and counts[0] > floor
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 10 * eps
    assert _rel(x, xd) <= 10 * eps
    assert _rel(x, xo) <= 10 * eps


# ---------------------------------------------------------------------------
# GMRES preconditioned by a loose factorization
# ---------------------------------------------------------------------------

def test_gmres_with_loose_factor_reaches_dense_accuracy(pkg, ell):
    s, A, b, xd = ell
    eps = 1e-2
    fac = pkg.Factorization(s.points, s.normals, s.weights, K, eps, leaf_size=24)
    try:
        c = np.conj(b[::-1]).copy()
        B2 = np.stack([b, c], axis=1)
        x, its, rel, ok = fac.gmres(torch.from_numpy(B2), tol=1e-12, restart=20, maxiter=60)
        x = x.cpu().numpy()
        # the step limit is reported, with the last iterate and its residual
        x1, its1, rel1, ok1 = fac.gmres(torch.from_numpy(b), tol=1e-14, restart=20, maxiter=1)
    finally:
        fac.free()
    assert ok and all(r <= 2e-12 for r in rel)
    assert _rel(x[:, 0], xd) <= 1e-10
    assert _rel(x[:, 1], dense.solve(A, c)) <= 1e-10
    for m in range(2):
        assert np.linalg.norm(A @ x[:, m] - B2[:, m]) / np.linalg.norm(B2[:, m]) <= 2e-12
    # the oracle's GMRES with its own factorization at the same eps
    F = rss.factor(s.points, s.normals, s.weights, K, eps, leaf_size=24)
    xo, its_o, hist = ogmres.gmres(lambda v: A @ v, lambda v: rss.solve(F, v), b, tol=1e-12,
                                   restart=20, maxiter=60)
    assert abs(its[0] - its_o) <= 1
    assert its[0] <= 10
    assert not ok1 and its1 == [1] and rel1[0] > 1e-14


# ---------------------------------------------------------------------------
# sonar cross section
# ---------------------------------------------------------------------------

def test_sonar_sweep_matches_oracle(pkg):
    s = synth.ellipsoid_graded_tip(3000, (1.0, 3.0, 0.5), seed=6)
    k, eps = 5.0, 1e-6
    phis = np.linspace(0.0, 2.0 * np.pi, 48, endpoint=False)
    dirs = sonar.azimuthal_directions(phis)
    A = kernel.dense_matrix(s.points, s.normals, s.weights, k, k)
    Bo = sonar.plane_wave_rhs(s.points, s.weights, k, dirs)
    Xd = dense.solve(A, Bo)
    Rd = sonar.backscatter(s.points, s.normals, s.weights, k, k, dirs, Xd)
    fac = pkg.Factorization(s.points, s.normals, s.weights, k, eps, leaf_size=32,
                            precision=pkg.PRECISION_FP64)
    try:
        R = fac.sonar_cross_section(phis, batch=16).cpu().numpy()
        # the two kernels alone, on the oracle's right-hand sides and solutions
        dt = torch.from_numpy(dirs).cuda()
        bt = torch.empty((48, s.n), dtype=torch.complex128, device="cuda")
        pkg.fmmlu_plane_waves(fac.points, fac.weights, k, dt, bt)
        Rt = torch.empty(48, dtype=torch.complex128, device="cuda")
        pkg.fmmlu_backscatter(fac.points, fac.normals, fac.weights, k, k, dt,
                              torch.from_numpy(np.ascontiguousarray(Xd.T)).cuda(), Rt)
        bg, Rg = bt.cpu().numpy().T, Rt.cpu().numpy()
    finally:
        fac.free()
    assert np.max(np.abs(bg - Bo)) <= 1e-14 * np.max(np.abs(Bo))
    assert np.max(np.abs(Rg - Rd)) <= 1e-12 * np.max(np.abs(Rd))
    assert np.max(np.abs(R - Rd)) <= 10 * eps * np.max(np.abs(Rd))
    F = rss.factor(s.points, s.normals, s.weights, k, eps, leaf_size=32)
    Ro = sonar.backscatter(s.points, s.normals, s.weights, k, k, dirs, rss.solve(F, Bo))
    assert np.max(np.abs(R - Ro)) <= 10 * eps * np.max(np.abs(Ro))
