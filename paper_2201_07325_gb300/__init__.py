"""GB300 FMM-LU: recursive strong skeletonization of the 3-D Helmholtz CFIE.

The compute path is libfmmlu.so (hand-written CUDA for sm_103a) behind the C ABI
of include/fmmlu.h; this package is its thin Python binding plus the
`Factorization` object and the `FMMLUSolve` autograd function.
"""
from .binding import (FmmluError, PRECISION_AUTO, PRECISION_FP64, PRECISION_MIXED,  # noqa: F401
                      ID_AUTO, ID_GRAM, ID_HOUSEHOLDER, PROXY_ADAPTIVE, PROXY_FIXED,
                      fmmlu_backscatter, fmmlu_gmres, fmmlu_plane_waves, fmmlu_solve_noalloc,
                      fmmlu_sonar_sweep, fmmlu_build_tree, fmmlu_default_opts, fmmlu_factor, fmmlu_free,
                      fmmlu_kernel_launches, fmmlu_last_error, fmmlu_matvec,
                      fmmlu_profile_reset, fmmlu_opts, fmmlu_solve,
                      fmmlu_solve_adjoint, fmmlu_stats, fmmlu_tree_describe, load_library,
                      parse_tree_description)
from .solver import FMMLUSolve, Factorization, fmmlu_solve_autograd  # noqa: F401
