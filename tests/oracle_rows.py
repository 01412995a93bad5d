"""Sampled rows and columns of the dense system, evaluated by the oracle in a
pool of worker processes (for residuals at sizes where A cannot be formed).

Test infrastructure. The pool is started with the `spawn` method, so it is
safe to use after the CUDA context of the test process exists (a pool forked
from a process that holds a CUDA context can hang). The arrays are handed to
the workers as .npy files opened memory-mapped, so each worker reads what it
needs instead of receiving pickled copies.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile
from concurrent.futures import ProcessPoolExecutor

import numpy as np


def _row_task(args):
    d, k, eta, rows = args
    from oracle import kernel
    x = np.load(os.path.join(d, "x.npy"), mmap_mode="r")
    nrm = np.load(os.path.join(d, "n.npy"), mmap_mode="r")
    w = np.load(os.path.join(d, "w.npy"), mmap_mode="r")
    v = np.load(os.path.join(d, "v.npy"), mmap_mode="r")
    return kernel.matvec(np.asarray(x), np.asarray(nrm), np.asarray(w), k, eta,
                         np.asarray(v), rows)


def _col_task(args):
    d, k, eta, cols, j0, j1 = args
    from oracle import kernel
    x = np.asarray(np.load(os.path.join(d, "x.npy"), mmap_mode="r"))
    nrm = np.asarray(np.load(os.path.join(d, "n.npy"), mmap_mode="r"))
    w = np.asarray(np.load(os.path.join(d, "w.npy"), mmap_mode="r"))
    v = np.load(os.path.join(d, "v.npy"), mmap_mode="r")
    out = 0
    step = max(1, 2_000_000 // max(1, len(cols)))
    for a in range(j0, j1, step):
        b = min(j1, a + step)
        blk = kernel.matrix_block(np.arange(a, b), cols, x, nrm, w, k, eta)
        out = out + blk.conj().T @ np.asarray(v[a:b])
    return out


def _pool(procs):
    return ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn"))


def _save(d, points, normals, weights, v):
    for name, arr in (("x", points), ("n", normals), ("w", weights), ("v", v)):
        np.save(os.path.join(d, name + ".npy"), np.ascontiguousarray(arr))


def workers() -> int:
    try:
        return max(1, min(16, len(os.sched_getaffinity(0))))
    except Exception:
        return max(1, min(16, os.cpu_count() or 1))


def rows_of_product(points, normals, weights, k, eta, v, rows, procs=None):
    """(A v)[rows] for v of shape (N,) or (N, nrhs), in parallel over rows."""
    procs = procs or workers()
    rows = np.asarray(rows, dtype=np.int64)
    parts = np.array_split(rows, max(1, min(len(rows), 4 * procs)))
    with tempfile.TemporaryDirectory() as d:
        _save(d, points, normals, weights, v)
        with _pool(procs) as ex:
            res = list(ex.map(_row_task, [(d, k, eta, p) for p in parts if p.size]))
    return np.concatenate(res, axis=0)


def rows_of_adjoint_product(points, normals, weights, k, eta, y, cols, procs=None):
    """(A^H y)[cols] = sum_j conj(A[j, cols]) y_j, in parallel over blocks of j."""
    procs = procs or workers()
    n = points.shape[0]
    cols = np.asarray(cols, dtype=np.int64)
    bounds = np.linspace(0, n, 4 * procs + 1).astype(np.int64)
    with tempfile.TemporaryDirectory() as d:
        _save(d, points, normals, weights, y)
        with _pool(procs) as ex:
            res = list(ex.map(_col_task, [(d, k, eta, cols, int(bounds[i]), int(bounds[i + 1]))
                                          for i in range(len(bounds) - 1)
                                          if bounds[i + 1] > bounds[i]]))
    return sum(res)
