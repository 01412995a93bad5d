"""CPU FP64 oracle for the FMM-LU hot path (test infrastructure only).

This package is the plain, slow reference the CUDA library is checked against.
It is test infrastructure: only the tests, the smoke check and the benchmark's
CPU-baseline leg may import it; the library and its binding never do. It shares
no code with the CUDA path.

Modules
  kernel  -- Green's function, combined-field kernel, dense system matrix with
             the disc self term (Sec. 3, Eqs. greenfunhelm, comb_ref, disc3)
  dense   -- dense LU solve of the full system (reference solution)
  tree    -- level-restricted adaptive octree, near/far lists, colouring (Sec. 4)
  rss     -- recursive strong skeletonization with proxy compression, the
             factor application and its adjoint (Sec. 4.1, 4.2, 5.1)

Pins (what each part is checked against, other than itself) are listed in the
module headers and exercised by tests/test_oracle_*.py.
"""

