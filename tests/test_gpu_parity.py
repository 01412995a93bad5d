"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Integer work (the octree, permutation, lists, colours) must match bit for bit.
Floating point: the factorization is an eps-accurate approximation with
several valid answers (skeleton choice at near-tied pivots), so results are
compared where they are unique -- the solution and the residual, which both
sides must reach within 10 eps of the dense solve (Sec. 6.1 protocol, target
residual 10 eps) -- and per-box ranks are compared where pivots are not tied.
Exact cases (eps -> 0, a single box) must match the dense LU to ~1e-10.
"""
import numpy as np
import pytest

import synth
from oracle import dense, kernel, rss
from oracle import tree as otree

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_07325_gb300 as p
    p.load_library()
    return p


def _cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


# ---------------------------------------------------------------------------
# octree: bit-exact
# ---------------------------------------------------------------------------

TREE_CASES = [
    ("sphere2k", lambda: synth.sphere_fibonacci(2000), 64),
    ("ellipsoid3k", lambda: synth.ellipsoid_uniform(3000, seed=13), 24),
    ("torus5k_graded", lambda: synth.torus_graded(5000, seed=5), 24),
    ("tip3k_graded", lambda: synth.ellipsoid_graded_tip(3000, seed=6), 16),
    ("tiny", lambda: synth.sphere_fibonacci(40), 64),
    ("one_point", lambda: synth.Surface(np.array([[0.3, -0.2, 0.1]]), np.array([[1.0, 0, 0]]),
                                        np.array([0.5])), 64),
]


@pytest.mark.parametrize("name,mk,ls", TREE_CASES, ids=[c[0] for c in TREE_CASES])
def test_tree_matches_oracle(pkg, name, mk, ls):
    s = mk()
    opts = pkg.fmmlu_default_opts(leaf_size=ls)
    t = pkg.fmmlu_build_tree(_cuda(s.points), opts)
    try:
        d = pkg.parse_tree_description(pkg.fmmlu_tree_describe(t))
    finally:
        pkg.fmmlu_free(t)
    T = otree.build_tree(s.points, ls)
    assert d["n"] == s.n
    assert d["perm"] == list(T.perm)
    assert d["nlevels"] == T.nlevels
    assert len(d["boxes"]) == len(T.boxes)
    for i, b in enumerate(T.boxes):
        assert d["boxes"][i] == (b.level, *b.cell, b.start, b.end, b.parent, len(b.children))
    for lev, L in T.levels.items():
        col, near, farq = d["levels"][lev]
        for B in L.boxes:
            assert col[B] == L.colour[B]
            assert near[B] == L.near[B]
            assert farq[B] == L.farq[B]


# ---------------------------------------------------------------------------
# dense on-the-fly product (kernel device functions)
# ---------------------------------------------------------------------------

def test_matvec_matches_dense(pkg):
    s = synth.ellipsoid_uniform(1500, seed=3)
    k = 3.7
    A = kernel.dense_matrix(s.points, s.normals, s.weights, k, k)
    rng = np.random.default_rng(1)
    v = rng.standard_normal((2, s.n)) + 1j * rng.standard_normal((2, s.n))
    y = torch.empty((2, s.n), dtype=torch.complex128, device="cuda")
    pkg.fmmlu_matvec(_cuda(s.points), _cuda(s.normals), _cuda(s.weights), k, k,
                     _cuda(v, torch.complex128), y)
    ref = (A @ v.T).T
    assert np.linalg.norm(y.cpu().numpy() - ref) <= 1e-13 * np.linalg.norm(ref)


# ---------------------------------------------------------------------------
# factorization + solve
# ---------------------------------------------------------------------------

K = 2.0 * np.pi


@pytest.fixture(scope="module")
def ell():
    s = synth.ellipsoid_uniform(2000, (1.0, 2.0, 0.5), seed=13)
    A = kernel.dense_matrix(s.points, s.normals, s.weights, K, K)
    b = synth.scaled_rhs(s, -synth.plane_wave(s.points, (0.0, 0.0, 1.0), K))
    return s, A, b, dense.solve(A, b)


def _gpu_factor(pkg, s, k, eps, **kw):
    return pkg.Factorization(s.points, s.normals, s.weights, k, eps, **kw)


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_solve_within_10eps_and_matches_oracle(pkg, ell, eps):
    s, A, b, xd = ell
    fac = _gpu_factor(pkg, s, K, eps, leaf_size=24, precision=pkg.PRECISION_FP64)
    x = fac.solve(torch.from_numpy(b)).cpu().numpy()
    st = fac.stats()
    fac.free()
    rec = []
    F = rss.factor(s.points, s.normals, s.weights, K, eps, leaf_size=24, record=rec)
    xo = rss.solve(F, b)
    res = np.linalg.norm(A @ x - b) / np.linalg.norm(b)
    assert res <= 10 * eps
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 10 * eps
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 10 * eps
    # compression happened on both sides, with comparable totals
    assert st["n0"] < s.n
    assert abs(st["n0"] - F.n0) <= max(10, 0.05 * F.n0)


def test_ranks_match_oracle(pkg, ell):
    s, A, b, xd = ell
    eps = 1e-6
    fac = _gpu_factor(pkg, s, K, eps, leaf_size=24, precision=pkg.PRECISION_FP64)
    st = fac.stats()
    fac.free()
    F = rss.factor(s.points, s.normals, s.weights, K, eps, leaf_size=24)
    for lev_stats in st["levels"]:
        lev = lev_stats["level"]
        L = F.tree.levels[lev]
        sum_a = sum(F.ranks[B][0] for B in L.boxes if B in F.ranks)
        sum_s = sum(F.ranks[B][1] for B in L.boxes if B in F.ranks)
        assert lev_stats["boxes"] == len(L.boxes)
        assert abs(lev_stats["sum_a"] - sum_a) <= max(2, 0.01 * sum_a)
        assert abs(lev_stats["sum_s"] - sum_s) <= max(2, 0.01 * sum_s)


def test_eps_to_zero_is_dense_lu(pkg, ell):
    s, A, b, xd = ell
    fac = _gpu_factor(pkg, s, K, 1e-14, leaf_size=24, precision=pkg.PRECISION_FP64)
    x = fac.solve(torch.from_numpy(b)).cpu().numpy()
    fac.free()
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-10


@pytest.mark.parametrize("emul", [0, 1, 2])
def test_schur_emulation_exact_limit_and_accuracy(pkg, ell, emul):
    """Elimination products in fp64 FMA (0), or on the bf16 tensor cores by
    exact operand splitting through tcgen05 with tensor-memory accumulators (1)
    or through mma.sync (2): eps -> 0 must still be the dense LU, eps = 1e-6
    within 10 eps, and every mode must agree with fp64 FMA far below eps."""
    s, A, b, xd = ell
    fac = _gpu_factor(pkg, s, K, 1e-14, leaf_size=24, precision=pkg.PRECISION_FP64,
                      schur_emulation=emul)
    x = fac.solve(torch.from_numpy(b)).cpu().numpy()
    fac.free()
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-10
    xs = {}
    for mode in sorted({0, emul}):
        fac = _gpu_factor(pkg, s, K, 1e-6, leaf_size=24, precision=pkg.PRECISION_FP64,
                          schur_emulation=mode)
        xs[mode] = fac.solve(torch.from_numpy(b)).cpu().numpy()
        fac.free()
    assert np.linalg.norm(A @ xs[emul] - b) / np.linalg.norm(b) <= 1e-5
    assert np.linalg.norm(xs[0] - xs[emul]) / np.linalg.norm(xs[0]) <= 1e-7


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gram_id_matches_householder_id(pkg, ell, prec):
    """The ID by pivoted Cholesky of G = M^H M (G formed exactly on the tensor
    cores) and by Householder CPQR of M make the same greedy selection (Def.
    ID) in exact arithmetic: per-level ranks agree up to near-tied pivots and
    both factorizations solve within 10 eps of the dense solution."""
    s, A, b, xd = ell
    eps = 1e-6 if prec == "fp64" else 1e-4
    P = pkg.PRECISION_FP64 if prec == "fp64" else pkg.PRECISION_MIXED
    out = {}
    for method, name in ((pkg.ID_HOUSEHOLDER, "householder"), (pkg.ID_GRAM, "gram")):
        fac = _gpu_factor(pkg, s, K, eps, leaf_size=24, precision=P, id_method=method)
        st = fac.stats()
        x = fac.solve(torch.from_numpy(b)).cpu().numpy()
        fac.free()
        assert st["id_method"] == name
        assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 10 * eps
        assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 10 * eps
        out[name] = st
    for lh, lg in zip(out["householder"]["levels"], out["gram"]["levels"]):
        assert lh["level"] == lg["level"] and lh["boxes"] == lg["boxes"]
        assert abs(lh["sum_s"] - lg["sum_s"]) <= max(2, 0.01 * lh["sum_s"])
    assert abs(out["householder"]["n0"] - out["gram"]["n0"]) <= max(4, 0.02 * out["gram"]["n0"])


@pytest.mark.parametrize("tol", [-1.0, 0.0, 1e-9])
def test_xrr_inverse_refinement_and_fallback(pkg, ell, tol):
    """X_RR^{-1} by an fp32 inverse plus Newton-Schulz steps on the tensor cores
    (tol 1e-9, the default), with every refined box inverted again in fp64
    (tol 0: the fallback path), and by fp64 Gauss-Jordan alone (tol < 0): each
    reproduces the dense LU at eps = 1e-14 and they agree far below eps = 1e-6."""
    s, A, b, xd = ell
    fac = _gpu_factor(pkg, s, K, 1e-14, leaf_size=24, precision=pkg.PRECISION_FP64,
                      xrr_refine_tol=tol)
    x = fac.solve(torch.from_numpy(b)).cpu().numpy()
    fac.free()
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-10
    xs = {}
    for t in sorted({-1.0, tol}):
        fac = _gpu_factor(pkg, s, K, 1e-6, leaf_size=24, precision=pkg.PRECISION_FP64,
                          xrr_refine_tol=t)
        xs[t] = fac.solve(torch.from_numpy(b)).cpu().numpy()
        st = fac.stats()
        fac.free()
        refined = sum(l["refined_inverses"] for l in st["levels"])
        fallbacks = sum(l["refine_fallbacks"] for l in st["levels"])
        if t < 0:
            assert refined == 0
        else:
            assert refined > 0
            assert fallbacks == (refined if t == 0.0 else 0)
    assert np.linalg.norm(A @ xs[tol] - b) / np.linalg.norm(b) <= 1e-5
    assert np.linalg.norm(xs[tol] - xs[-1.0]) / np.linalg.norm(xs[-1.0]) <= 1e-8


def test_single_box_is_dense_lu(pkg):
    s = synth.ellipsoid_uniform(50, seed=3)
    A = kernel.dense_matrix(s.points, s.normals, s.weights, 3.0, 3.0)
    b = synth.scaled_rhs(s, synth.plane_wave(s.points, (1, 0, 0), 3.0))
    fac = _gpu_factor(pkg, s, 3.0, 1e-6)
    assert fac.stats()["n0"] == 50
    x = fac.solve(torch.from_numpy(b)).cpu().numpy()
    y = fac.solve_adjoint(torch.from_numpy(b)).cpu().numpy()
    fac.free()
    assert np.linalg.norm(x - dense.solve(A, b)) <= 1e-12 * np.linalg.norm(x)
    assert np.linalg.norm(y - dense.solve_adjoint(A, b)) <= 1e-12 * np.linalg.norm(y)


def test_adjoint_dot_and_dense(pkg, ell):
    s, A, b, xd = ell
    fac = _gpu_factor(pkg, s, K, 1e-6, leaf_size=24, precision=pkg.PRECISION_FP64)
    rng = np.random.default_rng(7)
    c = rng.standard_normal(s.n) + 1j * rng.standard_normal(s.n)
    x = fac.solve(torch.from_numpy(b)).cpu().numpy()
    y = fac.solve_adjoint(torch.from_numpy(c)).cpu().numpy()
    fac.free()
    lhs, rhs = np.vdot(c, x), np.vdot(y, b)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    yd = dense.solve_adjoint(A, c)
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) <= 1e-5


def test_multiple_rhs_and_aliasing(pkg, ell):
    s, A, b, xd = ell
    fac = _gpu_factor(pkg, s, K, 1e-6, leaf_size=24)
    rng = np.random.default_rng(9)
    Bm = rng.standard_normal((3, s.n)) + 1j * rng.standard_normal((3, s.n))
    bt = torch.from_numpy(Bm).to("cuda")
    xt = torch.empty_like(bt)
    pkg.fmmlu_solve(fac.handle, bt, xt, s.n)
    xs = [fac.solve(torch.from_numpy(Bm[i])).cpu().numpy() for i in range(3)]
    inplace = bt.clone()
    pkg.fmmlu_solve(fac.handle, inplace, inplace, s.n)
    fac.free()
    for i in range(3):
        assert np.allclose(xt[i].cpu().numpy(), xs[i], rtol=0, atol=1e-13 * np.abs(xs[i]).max())
    assert torch.equal(inplace, xt)


def test_solve_graph_replay_and_chunk_sizes(pkg, ell):
    """The sweeps replayed as one CUDA graph give the eager launches' result
    bit for bit and count the same kernels; every chunk size of the C products
    gives the same solution up to the order of the partial sums."""
    s, A, b, xd = ell
    B2 = np.stack([b, np.conj(b)])
    bt = torch.from_numpy(B2).to("cuda")
    sols = {}
    for chunk in (16, 64, 4096):
        fac = _gpu_factor(pkg, s, K, 1e-6, leaf_size=24, precision=pkg.PRECISION_FP64,
                          solve_chunk=chunk, solve_graph=1)
        xs, ys, counts = [], [], []
        for _ in range(3):                 # eager, then captured, then replayed
            l0 = pkg.fmmlu_kernel_launches()
            x = torch.empty_like(bt)
            y = torch.empty_like(bt)
            pkg.fmmlu_solve(fac.handle, bt, x, s.n)
            pkg.fmmlu_solve_adjoint(fac.handle, bt, y, s.n)
            torch.cuda.synchronize()
            counts.append(pkg.fmmlu_kernel_launches() - l0)
            xs.append(x)
            ys.append(y)
        fac.free()
        assert torch.equal(xs[0], xs[1]) and torch.equal(xs[0], xs[2])
        assert torch.equal(ys[0], ys[1]) and torch.equal(ys[0], ys[2])
        assert counts[0] == counts[1] == counts[2] > 0
        sols[chunk] = (xs[0].cpu().numpy(), ys[0].cpu().numpy())
    x0, y0 = sols[64]
    for chunk, (x1, y1) in sols.items():
        assert np.linalg.norm(x1 - x0) <= 1e-11 * np.linalg.norm(x0), chunk
        assert np.linalg.norm(y1 - y0) <= 1e-11 * np.linalg.norm(y0), chunk
    res = np.linalg.norm(A @ x0[0] - b) / np.linalg.norm(b)
    assert res <= 1e-5


def test_solve_chunk_tuner_and_cache_file(pkg, ell, tmp_path):
    """autotune times the candidate chunks on the first solve, keeps the
    fastest, writes it to the cache file, and reuses it for a second handle of
    the same structure without timing again."""
    s, A, b, xd = ell
    path = tmp_path / "tune.txt"
    bt = torch.from_numpy(b).to("cuda")
    ref = _gpu_factor(pkg, s, K, 1e-6, leaf_size=24, precision=pkg.PRECISION_FP64,
                      solve_chunk=64)
    xr = ref.solve(bt).cpu().numpy()
    ref.free()
    for rep in range(2):
        fac = _gpu_factor(pkg, s, K, 1e-6, leaf_size=24, precision=pkg.PRECISION_FP64,
                          autotune=1, autotune_cache=str(path))
        x = fac.solve(bt).cpu().numpy()
        fac.free()
        assert np.linalg.norm(x - xr) <= 1e-11 * np.linalg.norm(xr)
        lines = [ln.split() for ln in path.read_text().splitlines()]
        solve = [ln for ln in lines if ln[0].startswith("solve_chunk|")]
        assert len(solve) == 1
        key, val = solve[0]
        assert key.endswith("|nrhs=1|adj=0")
        assert int(val) in (32, 64, 128, 256)
    with pytest.raises(pkg.FmmluError):
        _gpu_factor(pkg, s, K, 1e-6, leaf_size=24, solve_chunk=40)


def test_gram_chunk_tuning_is_exact(pkg, ell, tmp_path):
    """Every split-K chunk length of the Gram product adds the same exact
    integer digit products, so the factorization with the tuned chunk lengths
    equals the one with the fixed default bit for bit; the tuned choices go
    to the cache file."""
    s, A, b, xd = ell
    path = tmp_path / "tune.txt"
    bt = torch.from_numpy(b).to("cuda")
    xs = []
    for tune in (0, 1):
        fac = _gpu_factor(pkg, s, K, 1e-6, leaf_size=24, precision=pkg.PRECISION_FP64,
                          solve_chunk=64, autotune=tune,
                          autotune_cache=str(path) if tune else None)
        xs.append(fac.solve(bt))
        fac.free()
    torch.cuda.synchronize()
    assert torch.equal(xs[0], xs[1])
    lines = [ln.split() for ln in path.read_text().splitlines()]
    gram = [(key, int(val)) for key, val in lines if key.startswith("gram_chunk|")]
    assert gram and all(v in (32, 64, 128, 256, 4096) for _, v in gram)
    assert len({key for key, _ in gram}) == len(gram)


def test_mixed_precision_within_10eps(pkg, ell):
    s, A, b, xd = ell
    eps = 1e-4
    fac = _gpu_factor(pkg, s, K, eps, leaf_size=24, precision=pkg.PRECISION_MIXED)
    assert fac.stats()["precision"] == "mixed"
    x = fac.solve(torch.from_numpy(b)).cpu().numpy()
    fac.free()
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 10 * eps
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 10 * eps


def test_graded_torus_adaptive_tree(pkg):
    s = synth.torus_graded(3000, seed=5)
    k, eps = 5.0, 1e-4
    A = kernel.dense_matrix(s.points, s.normals, s.weights, k, k)
    b = synth.scaled_rhs(s, -synth.plane_wave(s.points, (0, 0, 1), k))
    fac = _gpu_factor(pkg, s, k, eps, leaf_size=24)
    x = fac.solve(torch.from_numpy(b)).cpu().numpy()
    fac.free()
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 10 * eps


def test_autograd_matches_dense_adjoint_and_fd(pkg):
    s = synth.sphere_fibonacci(1200)
    k, eps = 2.0, 1e-6
    A = kernel.dense_matrix(s.points, s.normals, s.weights, k, k)
    fac = _gpu_factor(pkg, s, k, eps, leaf_size=32, precision=pkg.PRECISION_FP64)
    dirs = synth.seeded_directions(3, 2204)
    Bm = np.stack([synth.scaled_rhs(s, -synth.plane_wave(s.points, d, k)) for d in dirs])
    amp = torch.tensor([1.0 + 0.5j, -0.3 + 0.2j, 0.7 - 0.1j], dtype=torch.complex128,
                       device="cuda", requires_grad=True)
    Bt = torch.from_numpy(Bm).to("cuda")
    t = synth.exterior_targets(20, 3.0)
    Kt = kernel.comb_kernel(t, s.points, s.normals, k, k) * np.sqrt(s.weights)[None, :]
    Ktt = torch.from_numpy(Kt).to("cuda")

    def loss_fn(a):
        b = (a[:, None] * Bt).sum(0)
        x = pkg.FMMLUSolve.apply(b, fac)
        u = Ktt @ x
        return (u.abs() ** 2).sum()

    L = loss_fn(amp)
    L.backward()
    g = amp.grad.detach().cpu().numpy()
    # dense reference: x = A^{-1} b, dL/dx = Kt^H Kt x, grad_b = A^{-H} dL/dx*
    a0 = amp.detach().cpu().numpy()
    b0 = (a0[:, None] * Bm).sum(0)
    x0 = dense.solve(A, b0)
    gx = Kt.conj().T @ (Kt @ x0)
    gb = dense.solve_adjoint(A, gx)
    gref = Bm.conj() @ gb
    # torch returns the conjugate Wirtinger gradient scaled by 2: dL/d(conj a) * 2
    assert np.linalg.norm(g - 2 * gref) <= 1e-6 * np.linalg.norm(gref) * 2 + 1e-5 * np.linalg.norm(g)
    # central finite differences in the real and imaginary directions
    h = 1e-6
    for j in range(3):
        for unit in (1.0, 1j):
            ap = amp.detach().clone(); ap[j] += h * unit
            am = amp.detach().clone(); am[j] -= h * unit
            fd = (loss_fn(ap).item() - loss_fn(am).item()) / (2 * h)
            an = (g[j].real if unit == 1.0 else g[j].imag)
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-6 * np.abs(g).max()
    fac.free()


def test_full_size_ellipsoid_sampled_residual(pkg):
    """The 50,000-point ellipsoid (k = 2 pi, eps = 1e-6) in the bench's launch
    configuration: residual on 1,500 sampled rows against the oracle's row
    evaluation, and the full residual through the dense GPU product."""
    s = synth.make_surface("ellipsoid50k")
    k, eps = synth.WORKLOADS["ellipsoid50k"]["k"], synth.WORKLOADS["ellipsoid50k"]["eps"]
    b = synth.make_rhs("ellipsoid50k", s)
    fac = _gpu_factor(pkg, s, k, eps)
    xg = fac.solve(torch.from_numpy(b))
    yg = fac.matvec(xg).cpu().numpy()
    x = xg.cpu().numpy()
    fac.free()
    assert np.linalg.norm(yg - b) / np.linalg.norm(b) <= 10 * eps
    rows = np.random.default_rng(0).choice(s.n, 1500, replace=False)
    r = kernel.matvec(s.points, s.normals, s.weights, k, k, x, rows) - b[rows]
    assert np.linalg.norm(r) / np.linalg.norm(b[rows]) <= 10 * eps


def test_invalid_arguments(pkg):
    s = synth.sphere_fibonacci(100)
    fac = _gpu_factor(pkg, s, 1.0, 1e-6)
    b = torch.zeros(100, dtype=torch.complex128, device="cuda")
    rc = pkg.load_library().fmmlu_solve(fac.handle, b.data_ptr(), b.data_ptr(), 0, None)
    assert rc == -1
    with pytest.raises(pkg.FmmluError):
        pkg.Factorization(s.points, s.normals, s.weights, 1.0, 2.0)
    bad = s.points.copy()
    bad[3, 1] = np.nan
    with pytest.raises(pkg.FmmluError):
        pkg.Factorization(bad, s.normals, s.weights, 1.0, 1e-6)
    fac.free()


@pytest.mark.parametrize("eps", [1e-6, 1e-14])
def test_tensor_core_sweeps_equal_double_float_sweeps(pkg, ell, eps):
    """With 16 right-hand sides and solve_tc_nrhs = 8 the products with the C
    blocks of the sweeps run on the tensor cores (exact split); they must
    agree with the double-float sweeps (solve_tc_nrhs = 0) to rounding, solve
    and adjoint, eager and replayed as a graph, and at eps -> 0 reproduce the
    dense solve."""
    s, A, b, xd = ell
    rng = np.random.default_rng(16)
    Bm = rng.standard_normal((16, s.n)) + 1j * rng.standard_normal((16, s.n))
    Bm[0] = b
    bt = torch.from_numpy(Bm).to("cuda")
    out = {}
    for tc in (8, 0):
        fac = _gpu_factor(pkg, s, K, eps, leaf_size=24, precision=pkg.PRECISION_FP64,
                          solve_tc_nrhs=tc)
        xs, ys = [], []
        for _ in range(3):                      # eager, captured, replayed
            x = torch.empty_like(bt)
            y = torch.empty_like(bt)
            pkg.fmmlu_solve(fac.handle, bt, x, s.n)
            pkg.fmmlu_solve_adjoint(fac.handle, bt, y, s.n)
            xs.append(x)
            ys.append(y)
        torch.cuda.synchronize()
        fac.free()
        assert torch.equal(xs[0], xs[1]) and torch.equal(xs[0], xs[2])
        assert torch.equal(ys[0], ys[1]) and torch.equal(ys[0], ys[2])
        out[tc] = (xs[0].cpu().numpy(), ys[0].cpu().numpy())
    for k in range(2):
        a, f = out[8][k], out[0][k]
        assert np.linalg.norm(a - f) <= 1e-12 * np.linalg.norm(f)
    if eps < 1e-10:
        assert np.linalg.norm(out[8][0][0] - xd) <= 1e-10 * np.linalg.norm(xd)
