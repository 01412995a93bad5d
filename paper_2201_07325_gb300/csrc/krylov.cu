// Preconditioned GMRES on the GPU (Sec. 7: the factorization at a loose
// tolerance used as a preconditioner for an iterative method).
//
// Right preconditioning, A M^{-1} u = b, x = M^{-1} u: M^{-1} is the stored
// factorization (the sweeps of solve.cu), A the dense on-the-fly product of
// assembly.cu. Each restart cycle orthonormalises the Krylov basis V of
// A M^{-1} by classical Gram-Schmidt applied twice (every pass: one kernel
// for the partial inner products of all basis vectors over blocks of rows,
// one that sums them in a fixed order, one update kernel), keeps the
// Hessenberg matrix triangular with Givens rotations (one single-thread
// kernel per step: the matrix is at most 65 x 64), and ends with the update
// x += M^{-1} (V y), y from the triangular system. All reductions use a fixed
// summation order, so a run is deterministic. The host reads one residual
// estimate per step to decide whether to stop.
#include <algorithm>

#include "device_common.cuh"

namespace fmmlu {

constexpr int kKrThreads = 256;

// part[blk * ncols + j] = sum over the block's rows i of conj(V[i, j]) w[i]
__global__ void __launch_bounds__(kKrThreads) k_kr_dots(const double2* __restrict__ V, int64_t ldv,
                                                        int ncols, const double2* __restrict__ w,
                                                        int64_t n, int64_t rows_per_blk,
                                                        double2* __restrict__ part) {
  __shared__ double2 red[kKrThreads / 32];
  const int64_t i0 = blockIdx.x * rows_per_blk;
  const int64_t i1 = min(n, i0 + rows_per_blk);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = 0; j < ncols; ++j) {
    const double2* vj = V + j * ldv;
    double2 acc = mk(0.0, 0.0);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) cfma_cj(acc, vj[i], w[i]);
    acc.x = warp_sum(acc.x);
    acc.y = warp_sum(acc.y);
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double2 s = red[0];
      for (int q = 1; q < kKrThreads / 32; ++q) s = cadd(s, red[q]);
      part[blockIdx.x * (int64_t)ncols + j] = s;
    }
    __syncthreads();
  }
}

// hc[j] = sum of the partials of column j (blocks in order); hacc[j] += hc[j]
// (the Hessenberg column over both Gram-Schmidt passes) unless hacc is null
__global__ void k_kr_dots_final(const double2* __restrict__ part, int nblk, int ncols,
                                double2* __restrict__ hc, double2* __restrict__ hacc) {
  const int j = threadIdx.x;
  if (j >= ncols) return;
  double2 s = mk(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) s = cadd(s, part[b * (int64_t)ncols + j]);
  hc[j] = s;
  if (hacc) hacc[j] = cadd(hacc[j], s);
}

// w -= V[:, 0:ncols] hc
__global__ void k_kr_update(double2* __restrict__ w, const double2* __restrict__ V, int64_t ldv,
                            int ncols, const double2* __restrict__ hc, int64_t n) {
  __shared__ double2 sh[kKrMaxBasis];
  for (int j = threadIdx.x; j < ncols; j += blockDim.x) sh[j] = hc[j];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 acc = w[i];
  for (int j = 0; j < ncols; ++j) cfms(acc, V[i + j * ldv], sh[j]);
  w[i] = acc;
}

// dst = src * scal[0] (scal holds 1/norm, 0 after a breakdown)
__global__ void k_kr_scale(double2* __restrict__ dst, const double2* __restrict__ src,
                           const double* __restrict__ scal, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = scal[0];
  dst[i] = mk(src[i].x * s, src[i].y * s);
}

// r = b - y
__global__ void k_kr_residual(double2* __restrict__ r, const double2* __restrict__ b,
                              const double2* __restrict__ y, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  r[i] = mk(b[i].x - y[i].x, b[i].y - y[i].y);
}

// x += z
__global__ void k_kr_add(double2* __restrict__ x, const double2* __restrict__ z, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = cadd(x[i], z[i]);
}

// u = V[:, 0:ncols] y
__global__ void k_kr_combine(double2* __restrict__ u, const double2* __restrict__ V, int64_t ldv,
                             int ncols, const double2* __restrict__ y, int64_t n) {
  __shared__ double2 sy[kKrMaxBasis];
  for (int j = threadIdx.x; j < ncols; j += blockDim.x) sy[j] = y[j];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 acc = mk(0.0, 0.0);
  for (int j = 0; j < ncols; ++j) acc = cadd(acc, cmul(V[i + j * ldv], sy[j]));
  u[i] = acc;
}

// One step's rotation (single thread): the norm of the orthogonalised vector
// completes column j of H; the earlier rotations are applied to it, a new
// one annihilates H[j+1, j], and the right-hand side g is rotated. est[0] =
// |g[j+1]| (the residual norm of the least-squares problem), est[1] = the
// norm; scal[0] = 1/norm (0 after a breakdown).
__global__ void k_kr_givens(double2* __restrict__ H, int ldh, int j,
                            const double2* __restrict__ nrm2, double* __restrict__ cs,
                            double2* __restrict__ sn, double2* __restrict__ g,
                            double* __restrict__ scal, double* __restrict__ est) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double hn = sqrt(fmax(nrm2[0].x, 0.0));
  double2* Hj = H + (int64_t)j * ldh;
  for (int i = 0; i < j; ++i) {
    const double2 a = Hj[i], b = Hj[i + 1];
    const double2 t = cadd(cscale(a, cs[i]), cmul(sn[i], b));
    Hj[i + 1] = csub(cscale(b, cs[i]), cmul(cconj(sn[i]), a));
    Hj[i] = t;
  }
  const double2 f = Hj[j];
  const double af = sqrt(cabs2(f));
  double c;
  double2 s, r;
  if (hn == 0.0) {
    c = 1.0; s = mk(0.0, 0.0); r = f;
  } else if (af == 0.0) {
    c = 0.0; s = mk(1.0, 0.0); r = mk(hn, 0.0);
  } else {
    const double nu = hypot(af, hn);
    const double2 ph = mk(f.x / af, f.y / af);
    c = af / nu;
    s = cscale(ph, hn / nu);          // (f/|f|) conj(hn) / nu, hn real
    r = cscale(ph, nu);
  }
  Hj[j] = r;
  Hj[j + 1] = mk(0.0, 0.0);
  cs[j] = c;
  sn[j] = s;
  const double2 gj = g[j];
  g[j + 1] = cmul(mk(-s.x, s.y), gj);  // -conj(s) g_j
  g[j] = cscale(gj, c);
  est[0] = sqrt(cabs2(g[j + 1]));
  est[1] = hn;
  scal[0] = hn > 0.0 ? 1.0 / hn : 0.0;
}

// start of a cycle: g = (beta, 0, ...), scal = 1/beta, est[0] = beta
__global__ void k_kr_start(const double2* __restrict__ nrm2, double2* __restrict__ g, int len,
                           double* __restrict__ scal, double* __restrict__ est) {
  const double beta = sqrt(fmax(nrm2[0].x, 0.0));
  for (int i = threadIdx.x; i < len; i += blockDim.x) g[i] = mk(i == 0 ? beta : 0.0, 0.0);
  if (threadIdx.x == 0) {
    scal[0] = beta > 0.0 ? 1.0 / beta : 0.0;
    est[0] = beta;
    est[1] = beta;
  }
}

// y = H[0:jd, 0:jd]^{-1} g[0:jd] (upper triangular, back substitution)
__global__ void k_kr_trisolve(const double2* __restrict__ H, int ldh, int jd,
                              const double2* __restrict__ g, double2* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = jd - 1; i >= 0; --i) {
    double2 acc = g[i];
    for (int l = i + 1; l < jd; ++l) cfms(acc, H[i + (int64_t)l * ldh], y[l]);
    y[i] = cdiv(acc, H[i + (int64_t)i * ldh]);
  }
}

// ---------------------------------------------------------------------------

static unsigned kr_grid(int64_t n) { return (unsigned)((n + kKrThreads - 1) / kKrThreads); }

int64_t kr_rows_per_block(int64_t n) {
  return std::max<int64_t>(4096, (n + 1023) / 1024);
}

int kr_blocks(int64_t n) { return (int)((n + kr_rows_per_block(n) - 1) / kr_rows_per_block(n)); }

void launch_kr_dots(const double2* V, int64_t ldv, int ncols, const double2* w, int64_t n,
                    double2* part, double2* hc, double2* hacc, cudaStream_t st) {
  const int64_t rpb = kr_rows_per_block(n);
  const int nblk = kr_blocks(n);
  FMMLU_LAUNCH("krylov_dots", st,
               k_kr_dots<<<nblk, kKrThreads, 0, st>>>(V, ldv, ncols, w, n, rpb, part));
  FMMLU_LAUNCH("krylov_small", st,
               k_kr_dots_final<<<1, kKrMaxBasis, 0, st>>>(part, nblk, ncols, hc, hacc));
}

void launch_kr_update(double2* w, const double2* V, int64_t ldv, int ncols, const double2* hc,
                      int64_t n, cudaStream_t st) {
  FMMLU_LAUNCH("krylov_vec", st,
               k_kr_update<<<kr_grid(n), kKrThreads, 0, st>>>(w, V, ldv, ncols, hc, n));
}

void launch_kr_scale(double2* dst, const double2* src, const double* scal, int64_t n,
                     cudaStream_t st) {
  FMMLU_LAUNCH("krylov_vec", st, k_kr_scale<<<kr_grid(n), kKrThreads, 0, st>>>(dst, src, scal, n));
}

void launch_kr_residual(double2* r, const double2* b, const double2* y, int64_t n,
                        cudaStream_t st) {
  FMMLU_LAUNCH("krylov_vec", st, k_kr_residual<<<kr_grid(n), kKrThreads, 0, st>>>(r, b, y, n));
}

void launch_kr_add(double2* x, const double2* z, int64_t n, cudaStream_t st) {
  FMMLU_LAUNCH("krylov_vec", st, k_kr_add<<<kr_grid(n), kKrThreads, 0, st>>>(x, z, n));
}

void launch_kr_combine(double2* u, const double2* V, int64_t ldv, int ncols, const double2* y,
                       int64_t n, cudaStream_t st) {
  FMMLU_LAUNCH("krylov_vec", st,
               k_kr_combine<<<kr_grid(n), kKrThreads, 0, st>>>(u, V, ldv, ncols, y, n));
}

void launch_kr_givens(double2* H, int ldh, int j, const double2* nrm2, double* cs, double2* sn,
                      double2* g, double* scal, double* est, cudaStream_t st) {
  FMMLU_LAUNCH("krylov_small", st,
               k_kr_givens<<<1, 32, 0, st>>>(H, ldh, j, nrm2, cs, sn, g, scal, est));
}

void launch_kr_start(const double2* nrm2, double2* g, int len, double* scal, double* est,
                     cudaStream_t st) {
  FMMLU_LAUNCH("krylov_small", st, k_kr_start<<<1, 64, 0, st>>>(nrm2, g, len, scal, est));
}

void launch_kr_trisolve(const double2* H, int ldh, int jd, const double2* g, double2* y,
                        cudaStream_t st) {
  FMMLU_LAUNCH("krylov_small", st, k_kr_trisolve<<<1, 32, 0, st>>>(H, ldh, jd, g, y));
}

}  // namespace fmmlu
