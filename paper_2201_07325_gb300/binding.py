"""ctypes binding of libfmmlu.so: the C-ABI entry points under the same names.

Argument marshalling only: every step of the method runs in the library's CUDA
kernels. Tensors passed in must be CUDA tensors of the right dtype and
contiguous layout; the functions take their data pointers and the current
torch CUDA stream. There is no CPU fallback: loading fails loudly when the
compiled library is missing.
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfmmlu.so")

ERRORS = {
    -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "SINGULAR_PIVOT",
    -5: "NONFINITE", -6: "DEPTH_CAP", -7: "TIMEOUT", -8: "LIMIT", -9: "NOT_CONVERGED",
}
PRECISION_AUTO, PRECISION_FP64, PRECISION_MIXED = 0, 1, 2
ID_AUTO, ID_HOUSEHOLDER, ID_GRAM = 0, 1, 2
PROXY_FIXED, PROXY_ADAPTIVE = 0, 1


class FmmluError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fmmlu error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class fmmlu_opts(ctypes.Structure):
    _fields_ = [
        ("leaf_size", ctypes.c_int),
        ("eta", ctypes.c_double),
        ("proxy_radius_factor", ctypes.c_double),
        ("n_proxy", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("eps_id_divisor", ctypes.c_double),
        ("verbose", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("cpqr_single", ctypes.c_int),
        ("schur_emulation", ctypes.c_int),
        ("id_method", ctypes.c_int),
        ("xrr_refine_tol", ctypes.c_double),
        ("solve_chunk", ctypes.c_int),
        ("solve_graph", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("autotune_cache", ctypes.c_char_p),
        ("solve_tc_nrhs", ctypes.c_int),
        ("proxy_rule", ctypes.c_int),
    ]


_lib = None


def load_library(path: str | None = None):
    """Load libfmmlu.so (build it first with paper_2201_07325_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(
            f"libfmmlu.so not found at {path}; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, i64, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    lib.fmmlu_default_opts.argtypes = [ctypes.POINTER(fmmlu_opts)]
    lib.fmmlu_default_opts.restype = ci
    lib.fmmlu_build_tree.argtypes = [vp, i64, ctypes.POINTER(fmmlu_opts), vp,
                                     ctypes.POINTER(vp)]
    lib.fmmlu_build_tree.restype = ci
    lib.fmmlu_factor.argtypes = [vp, vp, vp, vp, dbl, dbl, ctypes.POINTER(fmmlu_opts), vp,
                                 ctypes.POINTER(vp)]
    lib.fmmlu_factor.restype = ci
    lib.fmmlu_solve.argtypes = [vp, vp, vp, ci, vp]
    lib.fmmlu_solve.restype = ci
    lib.fmmlu_solve_adjoint.argtypes = [vp, vp, vp, ci, vp]
    lib.fmmlu_solve_adjoint.restype = ci
    lib.fmmlu_matvec.argtypes = [i64, vp, vp, vp, dbl, dbl, vp, vp, ci, vp]
    lib.fmmlu_matvec.restype = ci
    lib.fmmlu_stats.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.fmmlu_stats.restype = ci
    lib.fmmlu_tree_describe.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), i64]
    lib.fmmlu_tree_describe.restype = i64
    lib.fmmlu_kernel_launches.argtypes = []
    lib.fmmlu_kernel_launches.restype = i64
    lib.fmmlu_profile_reset.argtypes = [vp]
    lib.fmmlu_profile_reset.restype = ci
    lib.fmmlu_solve_noalloc.argtypes = [vp, vp, vp, ci, ci, vp]
    lib.fmmlu_solve_noalloc.restype = ci
    lib.fmmlu_gmres.argtypes = [vp, vp, vp, vp, vp, vp, ci, dbl, ci, ci,
                                ctypes.POINTER(ci), ctypes.POINTER(dbl), vp]
    lib.fmmlu_gmres.restype = ci
    lib.fmmlu_plane_waves.argtypes = [i64, vp, vp, dbl, vp, ci, vp, vp]
    lib.fmmlu_plane_waves.restype = ci
    lib.fmmlu_backscatter.argtypes = [i64, vp, vp, vp, dbl, dbl, vp, ci, vp, vp, vp]
    lib.fmmlu_backscatter.restype = ci
    lib.fmmlu_sonar_sweep.argtypes = [vp, vp, vp, vp, vp, ci, ci, vp, vp]
    lib.fmmlu_sonar_sweep.restype = ci
    lib.fmmlu_free.argtypes = [vp]
    lib.fmmlu_free.restype = None
    lib.fmmlu_last_error.argtypes = []
    lib.fmmlu_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise FmmluError(rc, load_library().fmmlu_last_error().decode())


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _cols(t: torch.Tensor, n: int, name: str):
    """complex128 (n,) or (n, nrhs) column-major view check -> (tensor, nrhs)."""
    _dev(t, torch.complex128, name)
    if t.dim() == 1:
        if t.shape[0] != n:
            raise ValueError(f"{name} must have length {n}")
        return t, 1
    if t.dim() == 2 and t.shape[1] == n:       # stored as (nrhs, n): column-major n x nrhs
        return t, t.shape[0]
    raise ValueError(f"{name} must be (n,) or (nrhs, n) (column-major n x nrhs)")


def fmmlu_default_opts(**overrides) -> fmmlu_opts:
    o = fmmlu_opts()
    _check(load_library().fmmlu_default_opts(ctypes.byref(o)))
    for k, v in overrides.items():
        if v is None:
            continue
        if not hasattr(o, k):
            raise KeyError(k)
        if k == "autotune_cache" and isinstance(v, str):
            v = v.encode()
        setattr(o, k, v)
    return o


def fmmlu_build_tree(points: torch.Tensor, opts: fmmlu_opts | None = None, stream=None):
    _dev(points, torch.float64, "points")
    out = ctypes.c_void_p()
    _check(load_library().fmmlu_build_tree(
        points.data_ptr(), points.shape[0], ctypes.byref(opts) if opts else None,
        _stream(stream), ctypes.byref(out)))
    return out


def fmmlu_factor(tree, points, normals, weights, k: float, eps: float,
                 opts: fmmlu_opts | None = None, stream=None):
    _dev(points, torch.float64, "points")
    _dev(normals, torch.float64, "normals")
    _dev(weights, torch.float64, "weights")
    out = ctypes.c_void_p()
    _check(load_library().fmmlu_factor(
        tree, points.data_ptr(), normals.data_ptr(), weights.data_ptr(), float(k), float(eps),
        ctypes.byref(opts) if opts else None, _stream(stream), ctypes.byref(out)))
    return out


def fmmlu_solve(handle, b: torch.Tensor, x: torch.Tensor, n: int, stream=None):
    b, nrhs = _cols(b, n, "b")
    x, nrhs2 = _cols(x, n, "x")
    if nrhs != nrhs2:
        raise ValueError("b and x must have the same number of columns")
    _check(load_library().fmmlu_solve(handle, b.data_ptr(), x.data_ptr(), nrhs,
                                      _stream(stream)))
    return x


def fmmlu_solve_adjoint(handle, b: torch.Tensor, x: torch.Tensor, n: int, stream=None):
    b, nrhs = _cols(b, n, "b")
    x, nrhs2 = _cols(x, n, "x")
    if nrhs != nrhs2:
        raise ValueError("b and x must have the same number of columns")
    _check(load_library().fmmlu_solve_adjoint(handle, b.data_ptr(), x.data_ptr(), nrhs,
                                              _stream(stream)))
    return x


def fmmlu_solve_noalloc(handle, b: torch.Tensor, x: torch.Tensor, n: int, adjoint: bool = False,
                        stream=None):
    """Solve (or adjoint solve) with the library's fixed work array: no
    device allocation; the call returns once the work is enqueued."""
    b, nrhs = _cols(b, n, "b")
    x, nrhs2 = _cols(x, n, "x")
    if nrhs != nrhs2:
        raise ValueError("b and x must have the same number of columns")
    _check(load_library().fmmlu_solve_noalloc(handle, b.data_ptr(), x.data_ptr(), nrhs,
                                              1 if adjoint else 0, _stream(stream)))
    return x


def fmmlu_matvec(points, normals, weights, k: float, eta: float, v: torch.Tensor,
                 y: torch.Tensor, stream=None):
    n = points.shape[0]
    _dev(points, torch.float64, "points")
    _dev(normals, torch.float64, "normals")
    _dev(weights, torch.float64, "weights")
    v, nrhs = _cols(v, n, "v")
    y, _ = _cols(y, n, "y")
    _check(load_library().fmmlu_matvec(n, points.data_ptr(), normals.data_ptr(),
                                       weights.data_ptr(), float(k), float(eta),
                                       v.data_ptr(), y.data_ptr(), nrhs, _stream(stream)))
    return y


def fmmlu_gmres(handle, points, normals, weights, b: torch.Tensor, x: torch.Tensor, n: int,
                tol: float = 1e-10, restart: int = 30, maxiter: int = 200, stream=None):
    """GMRES preconditioned by the factorization; returns (iters, relres,
    converged) with one entry of iters and relres per column."""
    _dev(points, torch.float64, "points")
    _dev(normals, torch.float64, "normals")
    _dev(weights, torch.float64, "weights")
    b, nrhs = _cols(b, n, "b")
    x, nrhs2 = _cols(x, n, "x")
    if nrhs != nrhs2:
        raise ValueError("b and x must have the same number of columns")
    its = (ctypes.c_int * nrhs)()
    rel = (ctypes.c_double * nrhs)()
    rc = load_library().fmmlu_gmres(handle, points.data_ptr(), normals.data_ptr(),
                                    weights.data_ptr(), b.data_ptr(), x.data_ptr(), nrhs,
                                    float(tol), int(restart), int(maxiter), its, rel,
                                    _stream(stream))
    if rc not in (0, -9):
        _check(rc)
    return list(its), list(rel), rc == 0


def _dirs(dirs: torch.Tensor) -> int:
    _dev(dirs, torch.float64, "dirs")
    if dirs.dim() != 2 or dirs.shape[1] != 3:
        raise ValueError("dirs must be (m, 3)")
    return int(dirs.shape[0])


def fmmlu_plane_waves(points, weights, k: float, dirs: torch.Tensor, b: torch.Tensor,
                      stream=None):
    """b (m, n) complex128 (column-major n x m) = -sqrt(w) exp(i k d_m . x)."""
    n = points.shape[0]
    _dev(points, torch.float64, "points")
    _dev(weights, torch.float64, "weights")
    m = _dirs(dirs)
    b, nb = _cols(b, n, "b")
    if nb != m:
        raise ValueError("b must have one column per direction")
    _check(load_library().fmmlu_plane_waves(n, points.data_ptr(), weights.data_ptr(), float(k),
                                            dirs.data_ptr(), m, b.data_ptr(), _stream(stream)))
    return b


def fmmlu_backscatter(points, normals, weights, k: float, eta: float, dirs: torch.Tensor,
                      x: torch.Tensor, R: torch.Tensor, stream=None):
    n = points.shape[0]
    for t, nm in ((points, "points"), (normals, "normals"), (weights, "weights")):
        _dev(t, torch.float64, nm)
    m = _dirs(dirs)
    x, nx = _cols(x, n, "x")
    _dev(R, torch.complex128, "R")
    if nx != m or R.numel() != m:
        raise ValueError("x and R must have one column / entry per direction")
    _check(load_library().fmmlu_backscatter(n, points.data_ptr(), normals.data_ptr(),
                                            weights.data_ptr(), float(k), float(eta),
                                            dirs.data_ptr(), m, x.data_ptr(), R.data_ptr(),
                                            _stream(stream)))
    return R


def fmmlu_sonar_sweep(handle, points, normals, weights, dirs: torch.Tensor, R: torch.Tensor,
                      batch: int = 64, stream=None):
    for t, nm in ((points, "points"), (normals, "normals"), (weights, "weights")):
        _dev(t, torch.float64, nm)
    m = _dirs(dirs)
    _dev(R, torch.complex128, "R")
    if R.numel() != m:
        raise ValueError("R must have one entry per direction")
    _check(load_library().fmmlu_sonar_sweep(handle, points.data_ptr(), normals.data_ptr(),
                                            weights.data_ptr(), dirs.data_ptr(), m, int(batch),
                                            R.data_ptr(), _stream(stream)))
    return R


def fmmlu_stats(handle) -> dict:
    lib = load_library()
    need = lib.fmmlu_stats(handle, None, 0)
    if need < 0:
        _check(need)
    buf = ctypes.create_string_buffer(need + 1)
    lib.fmmlu_stats(handle, buf, need + 1)
    return json.loads(buf.value.decode())


def fmmlu_tree_describe(tree):
    lib = load_library()
    need = lib.fmmlu_tree_describe(tree, None, 0)
    if need < 0:
        _check(int(need))
    arr = (ctypes.c_int64 * need)()
    lib.fmmlu_tree_describe(tree, arr, need)
    return list(arr)


def fmmlu_free(handle):
    if handle is not None and handle.value:
        load_library().fmmlu_free(handle)


def fmmlu_kernel_launches() -> int:
    return int(load_library().fmmlu_kernel_launches())


def fmmlu_profile_reset(handle):
    _check(load_library().fmmlu_profile_reset(handle))


def fmmlu_last_error() -> str:
    return load_library().fmmlu_last_error().decode()


def parse_tree_description(v):
    """Decode fmmlu_tree_describe output into plain Python structures."""
    n, nboxes, nlevels = v[0], v[1], v[2]
    p = 3
    boxes = []
    for _ in range(nboxes):
        boxes.append(tuple(v[p:p + 8]))
        p += 8
    perm = v[p:p + n]
    p += n
    levels = {}
    for lev in range(2, nlevels):
        ids = [i for i, b in enumerate(boxes) if b[0] == lev]
        col, near, farq = {}, {}, {}
        for B in ids:
            col[B] = v[p]
            nn = v[p + 1]
            near[B] = v[p + 2:p + 2 + nn]
            p += 2 + nn
            nq = v[p]
            farq[B] = v[p + 1:p + 1 + nq]
            p += 1 + nq
        levels[lev] = (col, near, farq)
    return dict(n=n, boxes=boxes, perm=perm, nlevels=nlevels, levels=levels)


__all__ = [
    "FmmluError", "fmmlu_opts", "load_library", "fmmlu_default_opts", "fmmlu_build_tree",
    "fmmlu_factor", "fmmlu_solve", "fmmlu_solve_adjoint", "fmmlu_matvec", "fmmlu_stats",
    "fmmlu_tree_describe", "fmmlu_free", "fmmlu_last_error", "parse_tree_description",
    "fmmlu_kernel_launches", "fmmlu_profile_reset", "fmmlu_solve_noalloc",
    "PRECISION_AUTO", "PRECISION_FP64", "PRECISION_MIXED", "ID_AUTO", "ID_HOUSEHOLDER", "ID_GRAM",
]

_ = math  # (kept for users composing eta = nan)
