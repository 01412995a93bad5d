/*
 * fmmlu.h -- C ABI of the GB300 FMM-LU library (recursive strong
 * skeletonization of the 3-D Helmholtz combined-field integral equation).
 *
 * The system solved is the sqrt(w)-scaled Nystrom discretisation of
 *     1/2 sigma + D sigma - i eta S sigma = f          (Sec. 3, Eq. disc3)
 * with G(x,y) = exp(i k |x-y|)/(4 pi |x-y|) (Eq. greenfunhelm) and the
 * combined-field kernel K(x,y) = n(y).grad_y G(x,y) - i eta G(x,y)
 * (Eq. comb_ref):
 *     A_ij = sqrt(w_i) K(x_i, x_j) sqrt(w_j)                     (i != j)
 *     A_ii = 1/2 - i eta (sqrt(w_i/pi)/2 + i k w_i/(4 pi))
 * The diagonal keeps the exterior jump 1/2, sets the double-layer self term
 * to 0 and replaces the single-layer self term by the two-term expansion of
 * the integral of G over a disc of area w_i. Right-hand sides are b = sqrt(w) f
 * and solutions x = sqrt(w) sigma.
 *
 * Conventions for every entry point:
 *  - Return 0 on success, a negative FMMLU_ERR_* code otherwise; the message
 *    of the last error of the calling thread is fmmlu_last_error(). No C++
 *    exception crosses this boundary; kernels never trap, they report through
 *    a device status word that the host turns into an error code.
 *  - Pointers documented "device" must be CUDA device (or managed) memory of
 *    the current device; "host" pointers are ordinary host memory.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). All work is
 *    ordered on it; calls that return sizes or statistics synchronise it.
 *  - Complex arrays are complex128, interleaved (re, im) doubles.
 *  - Point arrays are N x 3 row-major doubles in the caller's order. The
 *    library works in Morton order internally and permutes b and x itself.
 *  - The library copies what it needs from input arrays during the call; the
 *    caller keeps ownership of every array it passes. Handles own all their
 *    device memory (tree, factors) until fmmlu_free.
 */
#ifndef FMMLU_H
#define FMMLU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FMMLU_OK 0
#define FMMLU_ERR_INVALID_ARG -1  /* null pointer, n < 1, bad option value  */
#define FMMLU_ERR_OOM -2          /* a device or host allocation failed     */
#define FMMLU_ERR_CUDA -3         /* a CUDA runtime call failed             */
#define FMMLU_ERR_SINGULAR_PIVOT -4 /* X_RR or a root block had a zero or
                                       non-finite pivot (Sec. 4.1 assumes
                                       X_RR invertible)                      */
#define FMMLU_ERR_NONFINITE -5    /* NaN/Inf in inputs or in a computed ID   */
#define FMMLU_ERR_DEPTH_CAP -6    /* a leaf at the 21-level depth cap holds
                                     more than leaf_size points (warning
                                     only: reported by fmmlu_stats)          */
#define FMMLU_ERR_TIMEOUT -7      /* a bounded device wait gave up           */
#define FMMLU_ERR_LIMIT -8        /* a size exceeds a documented maximum     */
#define FMMLU_ERR_NOT_CONVERGED -9 /* an iteration stopped at its step limit
                                      before reaching its tolerance           */

#define FMMLU_ID_AUTO 0           /* Gram form when eps_ID >= 1e-7, else QR */
#define FMMLU_ID_HOUSEHOLDER 1    /* column-pivoted Householder QR of the ID
                                     matrix M                               */
#define FMMLU_ID_GRAM 2           /* pivoted Cholesky of G = M^H M, with G
                                     formed exactly on the tensor cores; its
                                     fp64 rounding is ~1e-16 |G|, so the
                                     rank rule resolves eps_ID down to about
                                     1e-7 (AUTO uses QR below that)         */
#define FMMLU_PRECISION_AUTO 0    /* mixed when eps >= 1e-5, else fp64       */
#define FMMLU_PRECISION_FP64 1    /* everything complex128                   */
#define FMMLU_PRECISION_MIXED 2   /* ID matrix assembly and pivoted QR in
                                     complex64 with fp32 accumulation; LU,
                                     Schur updates and apply stay complex128 */

typedef struct fmmlu_tree fmmlu_tree;
typedef struct fmmlu_handle fmmlu_handle;

/* Options. Fill with fmmlu_default_opts and change fields as needed. */
typedef struct fmmlu_opts {
  int leaf_size;              /* s of Sec. 4: split a box while it holds more
                                 than s points. Default 64. 1..4096          */
  double eta;                 /* coupling of -i eta S; NaN means eta = k     */
  double proxy_radius_factor; /* proxy sphere radius / box half-diagonal.
                                 Default 1.5; must lie in (1, 2.88) so the
                                 sphere encloses B and stays closer than
                                 2.5 h, inside which P never reaches       */
  int n_proxy;                /* proxy points per sphere (Fibonacci). 300   */
  int precision;              /* FMMLU_PRECISION_*                           */
  double eps_id_divisor;      /* ID tolerance eps_ID = eps / divisor. 1.0    */
  int verbose;                /* 0 quiet, 1 per-level lines on stderr        */
  int profile;                /* 1: time every kernel launch of the factor
                                 and of later solves with CUDA events on
                                 the launching stream and attribute the
                                 algorithmic flops/bytes to each kernel
                                 (reported by fmmlu_stats). Default 0.      */
  int cpqr_single;            /* 1: run every pivoted QR with one CTA per box
                                 (no row distribution). Default 0.          */
  int schur_emulation;        /* products of the elimination (G1, G3, X_RR,
                                 W, Schur update) and of the root, and the
                                 Gram matrix of the ID (every inner
                                 dimension in mode 1; >= 32 in mode 2,
                                 smaller ones on fp64 FMA):
                                 1 (default): tcgen05 tensor cores (TMEM
                                 accumulators) on an exact split of each
                                 complex128 operand into 7 bf16 digits; every
                                 digit product and partial sum is an exact
                                 integer, the only rounding is the final
                                 conversion to double;
                                 2: the same split on mma.sync tensor-core
                                 instructions (fp64 accumulation);
                                 0: fp64 FMA (Gram matrix as in 1). */
  int id_method;              /* FMMLU_ID_*: how the ID of Def. ID picks its
                                 skeleton (the same greedy column selection
                                 either way). Default FMMLU_ID_AUTO.        */
  double xrr_refine_tol;      /* schur_emulation 1 only: X_RR^{-1} of boxes
                                 with 32 <= r <= 640 is an fp32 inverse plus
                                 two or three Newton-Schulz steps on the
                                 tensor cores (the third is skipped where
                                 the second step's residual e gives
                                 (r e)^2 <= min(tol, eps/100)); a box whose
                                 last residual max|I - X_RR X| exceeds this
                                 tolerance is inverted again in fp64.
                                 Default 1e-9; 0 inverts every such box
                                 again; < 0 turns the refinement off (fp64
                                 Gauss-Jordan).                             */
  int solve_chunk;            /* rows of X_CR (forward sweep) and columns of
                                 X_RC (backward sweep) per CTA in the solves:
                                 0 (default) = chosen by the tuner when
                                 autotune = 1, else 64; otherwise a multiple
                                 of 16 in [16, 4096]. Results differ only in
                                 the order of partial sums.                 */
  int solve_graph;            /* 0: every solve launches its kernels;
                                 1 (default): the second and later solves
                                 with the same (nrhs, direction, stream)
                                 replay the sweeps as one CUDA graph;
                                 2: capture on the first solve. Solves with
                                 opts.profile = 1 never use graphs.        */
  int autotune;               /* 1 (default): pick launch schedules by
                                 timing them on the GPU, once per shape:
                                 - the split-K chunk length of each colour's
                                   Gram product (32, 64, 128, 256 or 4096
                                   k16 steps; every length gives the same
                                   exact sums), keyed by the colour's tile
                                   count and k range (log2 buckets);
                                 - with solve_chunk = 0, the solve chunk
                                   (32, 64, 128, 256) on the first solve
                                   with a given nrhs and direction, on the
                                   caller's right-hand sides.
                                 Results are shared by all handles in the
                                 process (and the cache file below).
                                 0: fixed defaults (128 steps; solve_chunk
                                 or 64).                                  */
  const char* autotune_cache; /* NULL or a file path: tuning results are read
                                 from it (lines "key value") and appended to
                                 it, so later processes skip the timing.
                                 The string is copied by fmmlu_factor.     */
  int solve_tc_nrhs;          /* solves with at least this many right-hand
                                 sides run the products with the C blocks
                                 (X_CR z in the forward sweep, X_RC x_C in
                                 the backward one, the bulk of the sweeps'
                                 arithmetic) on the tcgen05 tensor cores by
                                 the exact split of schur_emulation 1 (the
                                 operands split on every solve); fewer run
                                 on the CUDA cores in double-float
                                 arithmetic (every block entry read once per
                                 group of up to 8 right-hand sides).
                                 Default 32; 0 = never.                    */
  int proxy_rule;             /* number of proxy points per sphere (Sec. 5.2,
                                 proxy surface discretization):
                                 FMMLU_PROXY_FIXED (default): n_proxy on
                                 every level;
                                 FMMLU_PROXY_ADAPTIVE: per level from the
                                 multipole truncation estimate
                                 p = ceil(k rho + 1.8 d^(2/3) (k rho)^(1/3)),
                                 d = log10(1/eps_ID), rho the level's proxy
                                 radius: max(n_proxy, 2 (p + 1)^2) points, so
                                 n_proxy becomes the floor.                */
} fmmlu_opts;

#define FMMLU_PROXY_FIXED 0
#define FMMLU_PROXY_ADAPTIVE 1

/* Fill `opts` with the defaults listed above. Returns 0, or INVALID_ARG if
 * opts is NULL. */
int fmmlu_default_opts(fmmlu_opts* opts);

/* Build the level-restricted adaptive octree of Sec. 4 (preamble) and the
 * per-level near/far lists and colour classes of Sec. 4.2-4.3.
 *   points : device, N x 3 row-major doubles (caller order), read only
 *   n      : number of points, >= 1
 *   opts   : host, may be NULL (defaults)
 *   out    : host, receives a new tree handle (free with fmmlu_free)
 * Morton keys and the key sort run on the GPU; the box hierarchy, level
 * restriction (2:1 balance over face/edge/corner contacts), neighbour lists
 * and greedy colouring are built on the host from the sorted keys.
 * Errors: INVALID_ARG (null, n < 1, non-finite point), OOM, CUDA. */
int fmmlu_build_tree(const double* points, int64_t n, const fmmlu_opts* opts,
                     void* stream, fmmlu_tree** out);

/* Factor A (Sec. 4.2, RS-S with the proxy compression of Sec. 5.1).
 *   tree    : from fmmlu_build_tree on the same points
 *   points  : device, N x 3 (same array content as for the tree)
 *   normals : device, N x 3 unit outward normals
 *   weights : device, N positive quadrature weights
 *   k       : wavenumber (> 0); eta from opts (NaN -> k)
 *   eps     : ID tolerance in (0, 1): rank s = #{j : |R_jj| > eps |R_11|}
 *   out     : receives the factorization handle; all factors stay resident
 *             in device memory until fmmlu_free(handle)
 * The tree may be freed after this call. Errors: INVALID_ARG, OOM, CUDA,
 * SINGULAR_PIVOT, NONFINITE. */
int fmmlu_factor(const fmmlu_tree* tree, const double* points,
                 const double* normals, const double* weights, double k,
                 double eps, const fmmlu_opts* opts, void* stream,
                 fmmlu_handle** out);

/* x = A^{-1} b with the stored factors (Sec. 4.2, factored form of A^{-1}):
 * forward sweep in elimination order (E, L, D^{-1} per box), dense root
 * solve, backward sweep in reverse order (U, F per box).
 *   b, x : device, complex128, N x nrhs column-major (ld = N), caller order.
 *          b and x may be the same array. b is not modified otherwise.
 *   nrhs : >= 1
 * The call enqueues the work on `stream` and returns (with opts.profile = 1
 * it waits for it); order later reads of x on other streams after it.
 * Work vectors: the handle keeps those of the last four (nrhs, direction,
 * stream) combinations, about 16 nrhs (N + 2 n0) bytes plus partial sums
 * each, and their CUDA graphs (opts.solve_graph) until fmmlu_free. The first
 * solve with a new nrhs and direction may time the candidate chunk sizes
 * first (opts.autotune). Calls on one handle from several threads are
 * serialised on the host.
 * Errors: INVALID_ARG, OOM, CUDA. */
int fmmlu_solve(const fmmlu_handle* h, const double* b, double* x, int nrhs,
                void* stream);

/* x = A^{-H} b with the same factors (conjugate-transposed sweeps: the
 * forward sweep applies (F U)^H per box in elimination order, then the root
 * A_tt^{-H}, then the backward sweep (L E)^H per box in reverse order).
 * Same arguments and errors as fmmlu_solve. */
int fmmlu_solve_adjoint(const fmmlu_handle* h, const double* b, double* x,
                        int nrhs, void* stream);

/* y = A v with A assembled on the fly from the kernel (no factorization; an
 * independent dense product used for residuals). O(N^2) work.
 *   n    : number of points; points, normals, weights as for fmmlu_factor
 *          (device, caller order); eta NaN means eta = k;
 *   v, y : device complex128, N x nrhs column-major; y must not alias v.
 * Errors: INVALID_ARG, CUDA. */
int fmmlu_matvec(int64_t n, const double* points, const double* normals,
                 const double* weights, double k, double eta, const double* v,
                 double* y, int nrhs, void* stream);

/* Solve A x = b by restarted GMRES preconditioned by the stored factors:
 * the factorization used as a preconditioner for an iterative method
 * (Sec. 7). Right preconditioning, A M^{-1} u = b, x = M^{-1} u, with M^{-1}
 * the sweeps of fmmlu_solve and A the dense on-the-fly product of
 * fmmlu_matvec (O(N^2) per step). A factorization at a loose eps (fast, small
 * m_f) then reaches a tight tol in a few steps. Basis orthogonalised by
 * classical Gram-Schmidt applied twice, Givens rotations, x_0 = 0; every
 * step runs in the library's kernels; the host reads one residual estimate
 * per step.
 *   h       : the factorization (its N, k, eta define A)
 *   points, normals, weights : device, the arrays the factorization was
 *             computed from (caller order, as for fmmlu_factor)
 *   b, x    : device complex128, N x nrhs column-major; x must not alias b;
 *             each column is solved on its own
 *   tol     : in (0, 1): stop when the residual estimate <= tol ||b||
 *   restart : Krylov vectors per cycle, 1..64
 *   maxiter : total steps per column, >= 1
 *   iters   : host, nrhs ints (may be NULL): steps taken per column
 *   relres  : host, nrhs doubles (may be NULL): true ||b - A x|| / ||b||
 *             per column, from one more product after the last step
 * Synchronises the stream once per step. Work memory: (N x 69 + small)
 * complex128, allocated and freed by the call. Errors: INVALID_ARG, OOM,
 * CUDA, NOT_CONVERGED (some column's estimate stayed above tol; x, iters
 * and relres hold the last iterate). */
int fmmlu_gmres(const fmmlu_handle* h, const double* points, const double* normals,
                const double* weights, const double* b, double* x, int nrhs, double tol,
                int restart, int maxiter, int* iters, double* relres, void* stream);

/* Sound-soft boundary data of incident plane waves exp(i k d.x) (Sec. 6.3):
 * b[j + m N] = -sqrt(w_j) exp(i k d_m . x_j), the right-hand sides of the
 * sqrt(w)-scaled system for m = 0 .. m-1.
 *   points, weights : device, caller order (N x 3, N)
 *   dirs            : device, m x 3 row-major unit propagation directions
 *   b               : device complex128, N x m column-major (written)
 * Errors: INVALID_ARG, CUDA. */
int fmmlu_plane_waves(int64_t n, const double* points, const double* weights, double k,
                      const double* dirs, int m, double* b, void* stream);

/* Monostatic (backscattered) far-field pattern of the combined-field layer
 * potential of each column of x (Sec. 6.3, sonar cross section): for the
 * plane wave travelling along d_m, with u = e^{ikr}/r F + O(1/r^2),
 *   R_m = F(-d_m) = (1/(4 pi)) sum_j sqrt(w_j) x_{j,m} exp(i k d_m.x_j)
 *                   (i k n_j.d_m - i eta),
 * which for eta = k is (-i k/(4 pi)) sum_j sqrt(w_j) x_{j,m}
 * exp(i k d_m.x_j) (1 - n_j.d_m). x holds the solutions x~ = sqrt(w) sigma.
 *   points, normals, weights : device, caller order; eta NaN means k
 *   dirs : device, m x 3 row-major unit directions of incidence
 *   x    : device complex128, N x m column-major
 *   R    : device complex128, m values (written)
 * Synchronises the stream. Errors: INVALID_ARG, OOM, CUDA. */
int fmmlu_backscatter(int64_t n, const double* points, const double* normals,
                      const double* weights, double k, double eta, const double* dirs, int m,
                      const double* x, double* R, void* stream);

/* Sonar cross-section sweep (Sec. 6.3): for every direction d_m the plane
 * wave's right-hand side, the solve with the stored factors (batches of
 * `batch` right-hand sides per solve, at most 1024) and the backscattered
 * far field R_m as in fmmlu_backscatter, with the handle's k and eta.
 *   points, normals, weights : device, the factorization's arrays
 *   dirs  : device, m x 3 row-major unit directions (azimuthal sweep:
 *           d_m = (cos phi_m, sin phi_m, 0))
 *   R     : device complex128, m values (written)
 * Work memory N x batch complex128, allocated and freed by the call.
 * Synchronises the stream. Errors: INVALID_ARG, OOM, CUDA. */
int fmmlu_sonar_sweep(const fmmlu_handle* h, const double* points, const double* normals,
                      const double* weights, const double* dirs, int m, int batch, double* R,
                      void* stream);

/* Write a JSON object with the factorization statistics into `json` (host,
 * capacity `cap` bytes, always NUL-terminated when cap > 0): N, levels, n0,
 * factor bytes (m_f), per-level box counts, colours, rank sums, timings.
 * Returns the full length needed (excluding NUL), or a negative error code. */
int fmmlu_stats(const fmmlu_handle* h, char* json, size_t cap);

/* Write the tree as a flat int64 description into `out` (host, capacity
 * `cap` int64 values) for inspection: header {n, nboxes, nlevels}, then per
 * box {level, cx, cy, cz, start, end, parent, nchild}, then the Morton
 * permutation (N values), then per level >= 2 and per level box
 * {colour, n_near, near..., n_q, q...}. Returns the number of values needed,
 * or a negative error code. */
int64_t fmmlu_tree_describe(const fmmlu_tree* t, int64_t* out, int64_t cap);

/* Number of CUDA kernels this library has launched in the calling process
 * (all threads, all handles). Never fails. */
int64_t fmmlu_kernel_launches(void);

/* Clear the per-kernel accounting of a handle created with opts.profile = 1
 * (so that later solves can be measured alone). Returns 0 or INVALID_ARG. */
int fmmlu_profile_reset(const fmmlu_handle* h);

/* Size of the fixed device work array used by fmmlu_solve_noalloc. */
#define FMMLU_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* x = A^{-1} b (adjoint = 0) or x = A^{-H} b (adjoint != 0), the same sweeps
 * as fmmlu_solve / fmmlu_solve_adjoint, but without allocating any memory.
 * The paper has no counterpart: this entry point serves callers that cannot
 * call cudaMalloc while they solve -- for instance an application whose
 * device memory is handed out entirely by its own pool allocator (a
 * cudaMalloc would fail or bypass the pool), or a latency-critical loop that
 * must not pay the device-wide synchronisation of cudaFree.
 *   Work space: one fixed device array of FMMLU_NOALLOC_SCRATCH_BYTES (32 MiB)
 *   compiled into this library; every GPU that loads the library holds it
 *   until the process exits. A solve needs, each piece rounded up to 256 B,
 *     16 nrhs N                  (the permuted right-hand sides)
 *   + 2 x 16 nrhs n0             (the root's vectors)
 *   + 16 nrhs 64 ceil(n0/128) + 4 nrhs   (the root's partial sums)
 *   + 16 nrhs p                  (partial sums of the backward sweep)
 *   + 4 (boxes nrhs + 1)         (counters)
 *   bytes, where p is the largest sum over the boxes of one colour of
 *   r x (column chunks + 1) and can reach tens of times n0 with small
 *   chunks. fmmlu_stats reports the exact figure for nrhs = 1 as
 *   "noalloc_bytes" ({"solve": ..., "adjoint": ...}); larger requests return
 *   FMMLU_ERR_LIMIT and change nothing.
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture. The address is kept for the life of the
 *   process: after a cudaDeviceReset this entry point must not be used again.
 *   Device: call it with the device current that was current at
 *   fmmlu_factor (the one holding the factors); otherwise INVALID_ARG.
 *   Ordering: the call only enqueues work on `stream` and returns; synchronise
 *   the stream before reading x. All calls share the one array, which keeps
 *   the last call's contents (nothing in it needs to start at zero: the
 *   counters are cleared on the stream by every call): calls on one stream
 *   are ordered, calls that overlap on the GPU (other streams or threads)
 *   race.
 *   Profiling: with opts.profile = 1 the launches are timed like those of
 *   fmmlu_solve, the call waits for them, and fmmlu_stats counts them.
 *   b, x, nrhs as for fmmlu_solve. Errors: INVALID_ARG, LIMIT, CUDA. */
int fmmlu_solve_noalloc(const fmmlu_handle* h, const double* b, double* x, int nrhs,
                        int adjoint, void* stream);

/* Free a tree or a factorization handle (either kind; NULL is a no-op). */
void fmmlu_free(void* tree_or_handle);

/* Message of the last error on the calling thread ("" if none). */
const char* fmmlu_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FMMLU_H */
