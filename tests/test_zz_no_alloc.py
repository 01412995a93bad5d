"""fmmlu_solve_noalloc: the solve for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc while they solve -- an application whose
device memory is handed out entirely by its own pool allocator, or a
latency-critical loop that must not pay cudaFree's device-wide
synchronisation. fmmlu_solve_noalloc serves them from one fixed device array
inside the library. This test calls it through the C ABI twice in a row (the
array keeps the previous call's contents) for both the solve and the adjoint,
and compares each result with the allocating entry points fmmlu_solve and
fmmlu_solve_adjoint; it also checks that an oversized request is refused.
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_solve_matches_allocating_solve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_07325_gb300 as pkg
    lib = pkg.load_library()
    s = synth.ellipsoid_uniform(3000, (1.0, 2.0, 0.5), seed=31)
    k, eps = 2.0 * np.pi, 1e-6
    fac = pkg.Factorization(s.points, s.normals, s.weights, k, eps, leaf_size=32)
    try:
        dirs = synth.seeded_directions(2, 77)
        B = np.stack([synth.scaled_rhs(s, -synth.plane_wave(s.points, d, k)) for d in dirs])
        b = torch.from_numpy(B).to("cuda")                # (nrhs, n): column-major n x nrhs
        nrhs = b.shape[0]
        ref = torch.empty_like(b)
        ref_adj = torch.empty_like(b)
        pkg.fmmlu_solve(fac.handle, b, ref, s.n)
        pkg.fmmlu_solve_adjoint(fac.handle, b, ref_adj, s.n)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for adjoint, want in ((0, ref), (1, ref_adj)):
            for _ in range(2):                              # two calls in a row
                x = torch.full_like(b, complex(np.nan, np.nan))
                rc = lib.fmmlu_solve_noalloc(fac.handle, ctypes.c_void_p(b.data_ptr()),
                                             ctypes.c_void_p(x.data_ptr()), nrhs, adjoint,
                                             stream)
                assert rc == 0, pkg.fmmlu_last_error()
                torch.cuda.synchronize()
                err = torch.linalg.vector_norm(x - want) / torch.linalg.vector_norm(want)
                assert float(err) <= 1e-12
        # the statistics state the work space one right-hand side needs
        need = fac.stats()["noalloc_bytes"]
        assert 16 * s.n < need["solve"] <= 32 * 1024 * 1024
        assert 16 * s.n < need["adjoint"] <= 32 * 1024 * 1024
        # a request larger than the fixed array is refused and writes nothing
        big = 1 + (32 * 1024 * 1024) // (16 * s.n)
        bb = torch.ones((big, s.n), dtype=torch.complex128, device="cuda")
        xx = torch.zeros_like(bb)
        rc = lib.fmmlu_solve_noalloc(fac.handle, ctypes.c_void_p(bb.data_ptr()),
                                     ctypes.c_void_p(xx.data_ptr()), big, 0, stream)
        assert rc == -8 and "fixed array" in pkg.fmmlu_last_error()
        torch.cuda.synchronize()
        assert int(torch.count_nonzero(xx)) == 0
        # the shared array is still usable after the refusal
        x = torch.full_like(b, complex(np.nan, np.nan))
        rc = lib.fmmlu_solve_noalloc(fac.handle, ctypes.c_void_p(b.data_ptr()),
                                     ctypes.c_void_p(x.data_ptr()), nrhs, 0, stream)
        assert rc == 0, pkg.fmmlu_last_error()
        torch.cuda.synchronize()
        err = torch.linalg.vector_norm(x - ref) / torch.linalg.vector_norm(ref)
        assert float(err) <= 1e-12
    finally:
        fac.free()
