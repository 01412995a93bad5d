// Dense linear algebra of the factorization.
//
//  * k_cpqr      -- greedy column-pivoted Householder QR of the ID matrix
//                   (Def. ID; greedy CPQR as in Sec. 4.1): pivot = remaining
//                   column of largest norm (norms recomputed from the updated
//                   matrix, fused into the update), ties to the lowest index;
//                   stop when |R_jj| <= eps |R_11|; T = R_11^{-1} R_12. One CTA
//                   per box, one warp per column. fp32 or fp64.
//  * GEMM kernels (fp64 complex, 64x64 tiles) for Eq. strong-skel-elim:
//       G1[R,:] -= T^T G1[S,:]       (gives X_RS, X_RN and A_RR - T^T A_SR)
//       G3[:,R] -= G3[:,S] T         (gives X_SR, X_NR)
//       W = X_{CR} X_RR^{-1}
//       Delta[C,C] -= W X_{RC}       (Schur complement, scattered into the
//                                      per-box-pair Delta blocks)
//  * k_xrr_inverse -- X_RR = (A_RR - T^T A_SR) - X_RS T, then its inverse by
//                   Gauss-Jordan elimination with partial pivoting.
//  * root        -- block elimination of the remaining dense block: for each
//                   diagonal block D_i: D_i^{-1} (Gauss-Jordan), then
//                   A[later,later] -= A[later,i] D_i^{-1} A[i,later].
#include "device_common.cuh"

namespace fmmlu {

// ---------------------------------------------------------------------------
// CPQR
// ---------------------------------------------------------------------------

constexpr int kQrThreads = 512;

template <typename Rl>
__global__ void __launch_bounds__(kQrThreads) k_cpqr(LevelDev L, int b0) {
  using C = typename CT<Rl>::T;
  extern __shared__ unsigned char smem_raw[];
  int b = b0 + blockIdx.x;
  const BoxDesc d = L.desc[b];
  const int a = d.a;
  const int nq = L.run[b].nq;
  const int m = 2 * nq + 2 * L.n_proxy;
  const int64_t ld = d.mmax;
  C* M = reinterpret_cast<C*>(L.Mbuf) + d.M_off;
  Rl* norms = reinterpret_cast<Rl*>(smem_raw);
  int* perm = reinterpret_cast<int*>(norms + a);
  __shared__ int s_piv;
  __shared__ int s_rank;
  __shared__ Rl s_r11;
  __shared__ C s_v0, s_alpha;
  __shared__ Rl s_tau;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const Rl eps = (Rl)L.eps;

  for (int k = tid; k < a; k += blockDim.x) perm[k] = k;
  for (int k = warp; k < a; k += nw) {
    Rl acc = 0;
    for (int i = lane; i < m; i += 32) cnorm_acc(acc, M[i + k * ld]);
    acc = warp_sum(acc);
    if (lane == 0) norms[k] = acc;
  }
  if (tid == 0) s_rank = min(m, a);
  __syncthreads();
  const int steps = min(m, a);
  for (int j = 0; j < steps; ++j) {
    if (warp == 0) {
      Rl best = (Rl)-1;
      int bi = a;
      for (int k = j + lane; k < a; k += 32) {
        Rl v = norms[k];
        if (!(v == v)) v = (Rl)INFINITY;   // NaN: report below
        if (v > best) { best = v; bi = k; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        Rl ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        s_piv = bi;
        Rl nrm = sqrt(best);
        if (j == 0) s_r11 = nrm;
        if (!(nrm < (Rl)INFINITY)) set_status(L.status, kStatusNonfinite);
        if (!(nrm > eps * s_r11) || nrm == (Rl)0 || !(nrm < (Rl)INFINITY)) s_rank = j;
      }
    }
    __syncthreads();
    if (s_rank == j) break;
    const int p = s_piv;
    if (p != j) {
      for (int i = tid; i < m; i += blockDim.x) {
        C t = M[i + j * ld];
        M[i + j * ld] = M[i + p * ld];
        M[i + p * ld] = t;
      }
      if (tid == 0) {
        int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
        Rl tn = norms[j]; norms[j] = norms[p]; norms[p] = tn;
      }
    }
    __syncthreads();
    if (tid == 0) {
      C x0 = M[j + j * ld];
      Rl nx2 = norms[j];
      Rl nx = sqrt(nx2);
      Rl ax0 = sqrt(cabs2(x0));
      C ph = ax0 > (Rl)0 ? mk(x0.x / ax0, x0.y / ax0) : mk((Rl)1, (Rl)0);
      C alpha = mk(-ph.x * nx, -ph.y * nx);
      C v0 = csub(x0, alpha);
      Rl vv = nx2 - ax0 * ax0 + cabs2(v0);
      s_v0 = v0;
      s_alpha = alpha;
      s_tau = vv > (Rl)0 ? (Rl)2 / vv : (Rl)0;
    }
    __syncthreads();
    const C v0 = s_v0;
    const Rl tau = s_tau;
    for (int k = j + 1 + warp; k < a; k += nw) {
      C w = mk((Rl)0, (Rl)0);
      if (lane == 0) cfma_cj(w, v0, M[j + k * ld]);
      for (int i = j + 1 + lane; i < m; i += 32) cfma_cj(w, M[i + j * ld], M[i + k * ld]);
      w.x = warp_sum(w.x);
      w.y = warp_sum(w.y);
      C tw = mk(tau * w.x, tau * w.y);
      Rl acc = 0;
      if (lane == 0) {
        C t = M[j + k * ld];
        C u = cmul(v0, tw);
        M[j + k * ld] = csub(t, u);
      }
      for (int i = j + 1 + lane; i < m; i += 32) {
        C t = M[i + k * ld];
        cfms(t, M[i + j * ld], tw);
        M[i + k * ld] = t;
        cnorm_acc(acc, t);
      }
      acc = warp_sum(acc);
      if (lane == 0) norms[k] = acc;
    }
    __syncthreads();
    if (tid == 0) M[j + j * ld] = s_alpha;
    __syncthreads();
  }
  __syncthreads();
  const int s = s_rank;
  const int r = a - s;
  // T = R11^{-1} R12, in place in M[0:s, s:a] (column-oriented back substitution)
  for (int c = warp; c < r; c += nw) {
    C* col = M + (int64_t)(s + c) * ld;
    for (int i = s - 1; i >= 0; --i) {
      __syncwarp();
      C ti = cdiv(col[i], M[i + i * ld]);
      __syncwarp();
      if (lane == 0) col[i] = ti;
      for (int l = lane; l < i; l += 32) col[l] = csub(col[l], cmul(M[l + i * ld], ti));
    }
  }
  __syncthreads();
  double2* T = L.arena + d.T_off;
  for (int e = tid; e < s * r; e += blockDim.x) {
    int i = e % s, c = e / s;
    T[i + (int64_t)c * a] = to_d2(M[i + (int64_t)(s + c) * ld]);
  }
  // skeleton / redundant DOFs and the new active set of B
  int* idx = L.iarena + d.idx_off;
  int* pv = idx + a + d.nmax;
  const int base = L.cur_off[d.cur];
  const int* ndof = L.rows + d.rows_off + 3 * d.qmax;
  const int n = L.run[b].n;
  for (int k = tid; k < a; k += blockDim.x) {
    int p = perm[k];
    pv[k] = p;
    int dof = L.act_dof[base + p];
    if (k < s) idx[r + k] = dof; else idx[k - s] = dof;
    if (k < s) L.act_pos[base + k] = p;
  }
  for (int k = tid; k < n; k += blockDim.x) idx[a + k] = ndof[k];
  if (tid == 0) {
    L.run[b].s = s;
    L.run[b].r = r;
    L.cur_n[d.cur] = s;
  }
}

void launch_cpqr(const LevelDev& L, int b0, int nb, bool fp32, int amax, cudaStream_t st) {
  if (nb <= 0) return;
  if (fp32) {
    size_t sm = (size_t)amax * (sizeof(float) + sizeof(int));
    cudaFuncSetAttribute(k_cpqr<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    FMMLU_LAUNCH("cpqr", st, k_cpqr<float><<<nb, kQrThreads, sm, st>>>(L, b0));
  } else {
    size_t sm = (size_t)amax * (sizeof(double) + sizeof(int));
    cudaFuncSetAttribute(k_cpqr<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    FMMLU_LAUNCH("cpqr", st, k_cpqr<double><<<nb, kQrThreads, sm, st>>>(L, b0));
  }
}

// ---------------------------------------------------------------------------
// complex fp64 GEMM tile (64 x 64, 256 threads, 4 x 4 per thread)
// ---------------------------------------------------------------------------

constexpr int kTile = 64;
constexpr int kTk = 16;

struct GemmArgs {
  int m, n, k;
  const double2* A; int64_t lda;
  const double2* B; int64_t ldb;
};

// op(A)(i, kk): TA ? A[kk + i lda] : A[i + kk lda];  op(B)(kk, j): TB ? B[j + kk ldb] : B[kk + j ldb]
template <bool TA, bool TB, class Epi>
__device__ __forceinline__ void gemm_tile(const GemmArgs& g, int tm, int tn, Epi& epi) {
  __shared__ double2 As[kTk][kTile + 1];
  __shared__ double2 Bs[kTk][kTile + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int i0 = tm * kTile, j0 = tn * kTile;
  double2 acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = mk(0.0, 0.0);
  for (int k0 = 0; k0 < g.k; k0 += kTk) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int lin = tid + e * 256;
      int ii, kk;
      if (TA) { kk = lin & 15; ii = lin >> 4; } else { ii = lin & 63; kk = lin >> 6; }
      int gi = i0 + ii, gk = k0 + kk;
      double2 v = mk(0.0, 0.0);
      if (gi < g.m && gk < g.k) v = TA ? g.A[gk + gi * g.lda] : g.A[gi + gk * g.lda];
      As[kk][ii] = v;
      int jj;
      if (TB) { jj = lin & 63; kk = lin >> 6; } else { kk = lin & 15; jj = lin >> 4; }
      int gj = j0 + jj;
      gk = k0 + kk;
      double2 u = mk(0.0, 0.0);
      if (gj < g.n && gk < g.k) u = TB ? g.B[gj + gk * g.ldb] : g.B[gk + gj * g.ldb];
      Bs[kk][jj] = u;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kTk; ++kk) {
      double2 av[4], bv[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) av[p] = As[kk][ty + 16 * p];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) cfma(acc[p][q], av[p], bv[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int i = i0 + ty + 16 * p, j = j0 + tx + 16 * q;
      if (i < g.m && j < g.n) epi(i, j, acc[p][q]);
    }
}

struct EpiSub {   // C -= acc
  double2* C; int64_t ldc;
  __device__ void operator()(int i, int j, double2 v) {
    double2* c = C + i + j * ldc;
    *c = csub(*c, v);
  }
};
struct EpiStore {
  double2* C; int64_t ldc;
  __device__ void operator()(int i, int j, double2 v) { C[i + j * ldc] = v; }
};

__device__ __forceinline__ bool tile_of(int m, int n, int& tm, int& tn) {
  int tms = (m + kTile - 1) / kTile, tns = (n + kTile - 1) / kTile;
  int t = blockIdx.x;
  if (t >= tms * tns || m <= 0 || n <= 0) return false;
  tm = t % tms; tn = t / tms;
  return true;
}

// G1[s:a, :] -= T^T G1[0:s, :]     (r x (a+n), k = s)
__global__ void __launch_bounds__(256) k_gemm_g1(LevelDev L, int b0, int kskip) {
  int b = b0 + blockIdx.y;
  const BoxDesc d = L.desc[b];
  const BoxRun run = L.run[b];
  int a = d.a, s = run.s, r = run.r, n = run.n;
  if (r == 0 || s == 0 || (kskip > 0 && s >= kskip)) return;
  int tm, tn;
  if (!tile_of(r, a + n, tm, tn)) return;
  double2* G1 = L.arena + d.G1_off;
  GemmArgs g{r, a + n, s, L.arena + d.T_off, a, G1, a};
  EpiSub e{G1 + s, a};
  gemm_tile<true, false>(g, tm, tn, e);
}

// G3[:, s:a] -= G3[:, 0:s] T       ((a+n) x r, k = s)
__global__ void __launch_bounds__(256) k_gemm_g3(LevelDev L, int b0, int kskip) {
  int b = b0 + blockIdx.y;
  const BoxDesc d = L.desc[b];
  const BoxRun run = L.run[b];
  int a = d.a, s = run.s, r = run.r, n = run.n;
  if (r == 0 || s == 0 || (kskip > 0 && s >= kskip)) return;
  int tm, tn;
  if (!tile_of(a + n, r, tm, tn)) return;
  int64_t ld3 = a + d.nmax;
  double2* G3 = L.arena + d.G3_off;
  GemmArgs g{a + n, r, s, G3, ld3, L.arena + d.T_off, a};
  EpiSub e{G3 + s * ld3, ld3};
  gemm_tile<false, false>(g, tm, tn, e);
}

// W = X_CR Xinv       ((s+n) x r, k = r)
__global__ void __launch_bounds__(256) k_gemm_w(LevelDev L, int b0, int kskip) {
  int b = b0 + blockIdx.y;
  const BoxDesc d = L.desc[b];
  const BoxRun run = L.run[b];
  int a = d.a, s = run.s, r = run.r, n = run.n;
  if (r == 0 || (kskip > 0 && r >= kskip)) return;
  int tm, tn;
  if (!tile_of(s + n, r, tm, tn)) return;
  int64_t ld3 = a + d.nmax;
  GemmArgs g{s + n, r, r, L.arena + d.G3_off + s * ld3, ld3, L.arena + d.Xinv_off, a};
  EpiStore e{L.Wbuf + d.W_off, ld3};
  gemm_tile<false, false>(g, tm, tn, e);
}

// Delta[C, C] -= W X_RC    ((s+n) x (s+n), k = r), scattered into pair blocks
struct EpiSchur {
  const LevelDev* L;
  const BoxDesc* d;
  const int* rloc; const int* rpos;   // per tile row (shared)
  const int* cloc; const int* cpos;   // per tile col (shared)
  int i0, j0;
  __device__ void operator()(int i, int j, double2 v) {
    int li = rloc[i - i0], lj = cloc[j - j0];
    int cnt = 1 + d->ncnt;
    int64_t off = L->pairtab[d->pairtab + (int64_t)li * cnt + lj];
    if (off < 0) { set_status(L->status, kStatusBound); return; }
    int ld = li == 0 ? d->a : L->cur_a0[L->nlist[d->nbeg + li - 1]];
    double2* p = L->delta + off + rpos[i - i0] + (int64_t)cpos[j - j0] * ld;
    *p = csub(*p, v);
  }
};

__global__ void __launch_bounds__(256) k_schur(LevelDev L, int b0, int kskip) {
  __shared__ int rloc[kTile], rpos[kTile], cloc[kTile], cpos[kTile];
  int b = b0 + blockIdx.y;
  const BoxDesc d = L.desc[b];
  const BoxRun run = L.run[b];
  int a = d.a, s = run.s, r = run.r, n = run.n;
  if (r == 0 || (kskip > 0 && r >= kskip)) return;
  int tm, tn;
  if (!tile_of(s + n, s + n, tm, tn)) return;
  const int* perm = L.iarena + d.idx_off + a + d.nmax;
  const int* ndof = L.rows + d.rows_off + 3 * d.qmax;
  const int* npos = ndof + d.nmax;
  const int* nloc = npos + d.nmax;
  int i0 = tm * kTile, j0 = tn * kTile;
  if (threadIdx.x < kTile) {
    int t = threadIdx.x;
    int i = i0 + t;
    if (i < s) { rloc[t] = 0; rpos[t] = perm[i]; }
    else if (i < s + n) { rloc[t] = nloc[i - s]; rpos[t] = npos[i - s]; }
    int j = j0 + t;
    if (j < s) { cloc[t] = 0; cpos[t] = perm[j]; }
    else if (j < s + n) { cloc[t] = nloc[j - s]; cpos[t] = npos[j - s]; }
  }
  __syncthreads();
  int64_t ld3 = a + d.nmax;
  GemmArgs g{s + n, s + n, r, L.Wbuf + d.W_off, ld3, L.arena + d.G1_off + s, a};
  EpiSchur e{&L, &d, rloc, rpos, cloc, cpos, i0, j0};
  gemm_tile<false, false>(g, tm, tn, e);
}

static inline unsigned tiles(int m, int n) {
  return (unsigned)(((m + kTile - 1) / kTile) * ((n + kTile - 1) / kTile));
}

void launch_gemm_g1(const LevelDev& L, int b0, int nb, int amax, int nmax_max,
                    cudaStream_t st, int kskip) {
  if (nb <= 0) return;
  FMMLU_LAUNCH("gemm_g1", st,
               k_gemm_g1<<<dim3(tiles(amax, 2 * amax + nmax_max), nb), 256, 0, st>>>(L, b0, kskip));
}

void launch_gemm_g3(const LevelDev& L, int b0, int nb, int amax, int nmax_max,
                    cudaStream_t st, int kskip) {
  if (nb <= 0) return;
  FMMLU_LAUNCH("gemm_g3", st,
               k_gemm_g3<<<dim3(tiles(amax + nmax_max, amax), nb), 256, 0, st>>>(L, b0, kskip));
}

void launch_gemm_w(const LevelDev& L, int b0, int nb, int amax, int nmax_max, cudaStream_t st,
                   int kskip) {
  if (nb <= 0) return;
  FMMLU_LAUNCH("gemm_w", st,
               k_gemm_w<<<dim3(tiles(amax + nmax_max, amax), nb), 256, 0, st>>>(L, b0, kskip));
}

void launch_schur_update(const LevelDev& L, int b0, int nb, int amax, int nmax_max,
                         cudaStream_t st, int kskip) {
  if (nb <= 0) return;
  FMMLU_LAUNCH("schur_update", st,
               k_schur<<<dim3(tiles(amax + nmax_max, amax + nmax_max), nb), 256, 0, st>>>(L, b0, kskip));
}

// ---------------------------------------------------------------------------
// Gauss-Jordan inverse with partial pivoting (in place, column-major, ld)
// ---------------------------------------------------------------------------

__device__ void gauss_jordan(double2* X, int r, int64_t ld, int* ipiv, int* status) {
  __shared__ int s_p;
  __shared__ double2 s_inv;
  __shared__ double s_best[32];
  __shared__ int s_bi[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < r; ++j) {
    // pivot search over rows j..r-1 of column j
    double best = -1.0;
    int bi = r;
    for (int i = j + tid; i < r; i += blockDim.x) {
      double v = cabs2(X[i + j * ld]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { s_best[warp] = best; s_bi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bb = s_best[0];
      int ib = s_bi[0];
      for (int w = 1; w < nw; ++w)
        if (s_best[w] > bb || (s_best[w] == bb && s_bi[w] < ib)) { bb = s_best[w]; ib = s_bi[w]; }
      s_p = ib;
      ipiv[j] = ib;
      if (!(bb > 0.0) || !(bb < INFINITY)) set_status(status, kStatusSingular);
    }
    __syncthreads();
    int p = s_p;
    if (p >= r) return;
    if (p != j)
      for (int c = tid; c < r; c += blockDim.x) {
        double2 t = X[j + c * ld];
        X[j + c * ld] = X[p + c * ld];
        X[p + c * ld] = t;
      }
    __syncthreads();
    if (tid == 0) {
      s_inv = cdiv(mk(1.0, 0.0), X[j + j * ld]);
      X[j + j * ld] = mk(1.0, 0.0);
    }
    __syncthreads();
    double2 inv = s_inv;
    for (int c = tid; c < r; c += blockDim.x) X[j + c * ld] = cmul(X[j + c * ld], inv);
    __syncthreads();
    // eliminate column j from the other rows: row i -= f_i * row j
    for (int e = tid; e < r * r; e += blockDim.x) {
      int i = e % r, c = e / r;
      if (i == j || c == j) continue;
      double2 f = X[i + j * ld];
      double2 xv = X[i + c * ld];
      cfms(xv, f, X[j + c * ld]);
      X[i + c * ld] = xv;
    }
    __syncthreads();
    for (int i = tid; i < r; i += blockDim.x) {
      if (i == j) continue;
      double2 f = X[i + j * ld];
      X[i + j * ld] = csub(mk(0.0, 0.0), cmul(f, X[j + j * ld]));
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int j = r - 1; j >= 0; --j) {
    int p = ipiv[j];
    if (p != j)
      for (int i = tid; i < r; i += blockDim.x) {
        double2 t = X[i + j * ld];
        X[i + j * ld] = X[i + p * ld];
        X[i + p * ld] = t;
      }
    __syncthreads();
  }
}

// X_RR = (A_RR - T^T A_SR) - X_RS T = G1[s:a, s+n:a+n] - G1[s:a, 0:s] T   (r x r, k = s)
struct EpiDiff {   // C = Y - acc
  double2* C; int64_t ldc;
  const double2* Y; int64_t ldy;
  __device__ void operator()(int i, int j, double2 v) { C[i + j * ldc] = csub(Y[i + j * ldy], v); }
};

__global__ void __launch_bounds__(256) k_gemm_xrr(LevelDev L, int b0, int kskip) {
  int b = b0 + blockIdx.y;
  const BoxDesc d = L.desc[b];
  const BoxRun run = L.run[b];
  int a = d.a, s = run.s, r = run.r, n = run.n;
  if (r == 0 || (kskip > 0 && s >= kskip)) return;
  int tm, tn;
  if (!tile_of(r, r, tm, tn)) return;
  const double2* G1 = L.arena + d.G1_off;
  GemmArgs g{r, r, s, G1 + s, a, L.arena + d.T_off, a};
  EpiDiff e{L.arena + d.Xinv_off, a, G1 + s + (int64_t)(s + n) * a, a};
  gemm_tile<false, false>(g, tm, tn, e);
}

__global__ void __launch_bounds__(512) k_xrr_inverse(LevelDev L, int b0, int skip_lo, int skip_hi) {
  extern __shared__ int ipiv[];
  int b = b0 + blockIdx.x;
  const BoxDesc d = L.desc[b];
  const BoxRun run = L.run[b];
  int r = run.r;
  if (r == 0 || (r >= skip_lo && r <= skip_hi)) return;   // refined on the tensor cores
  gauss_jordan(L.arena + d.Xinv_off, r, d.a, ipiv, L.status);
}

void launch_gemm_xrr(const LevelDev& L, int b0, int nb, int amax, cudaStream_t st, int kskip) {
  if (nb <= 0) return;
  FMMLU_LAUNCH("gemm_xrr", st,
               k_gemm_xrr<<<dim3(tiles(amax, amax), nb), 256, 0, st>>>(L, b0, kskip));
}

void launch_xrr_inverse(const LevelDev& L, int b0, int nb, int amax, cudaStream_t st,
                        int skip_lo, int skip_hi) {
  if (nb <= 0) return;
  FMMLU_LAUNCH("xrr_inverse", st,
               k_xrr_inverse<<<nb, 512, (size_t)amax * sizeof(int), st>>>(L, b0, skip_lo, skip_hi));
}

// Boxes refined by Newton-Schulz whose residual max |I - X_RR X_1| exceeds thr
// (the second iterate's error is about its square) are inverted again in
// fp64 from the stored copy of X_RR.
__global__ void __launch_bounds__(512) k_ns_fallback(LevelDev L, int b0,
                                                     const TcUnit* __restrict__ units, double thr) {
  extern __shared__ int ipiv[];
  const int b = b0 + units[blockIdx.x].box;
  const BoxDesc d = L.desc[b];
  const int r = L.run[b].r;
  const double err = __longlong_as_double((long long)L.ns_err[b]);
  if (r == 0 || err <= thr) return;
  double2* X = L.arena + d.Xinv_off;
  const double2* A = L.nsbuf + L.ns_off[b];
  for (int64_t e = threadIdx.x; e < (int64_t)r * r; e += blockDim.x) {
    const int i = (int)(e % r), c = (int)(e / r);
    X[i + (int64_t)c * d.a] = A[i + (int64_t)c * d.a];
  }
  __syncthreads();
  gauss_jordan(X, r, d.a, ipiv, L.status);
}

__global__ void k_ns_flag(LevelDev L, int b0, const TcUnit* __restrict__ units, int nunits,
                          double thr, unsigned char* skip) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= nunits) return;
  const int b = b0 + units[u].box;
  const double r = (double)L.run[b].r;
  const double e = __longlong_as_double((long long)L.ns_err[b]);
  const double bound = (r * e) * (r * e);
  const bool done = bound <= thr;   // false for NaN
  skip[b] = done ? 1 : 0;
  if (done) L.ns_err[b] = 0ull;     // the fallback test passes on the bound
}

void launch_ns_flag(const LevelDev& L, int b0, const TcUnit* d_units, int nunits, double thr,
                    unsigned char* skip, cudaStream_t st) {
  if (nunits <= 0) return;
  FMMLU_LAUNCH("xrr_fallback", st,
               k_ns_flag<<<(nunits + 127) / 128, 128, 0, st>>>(L, b0, d_units, nunits, thr, skip));
}

void launch_ns_fallback(const LevelDev& L, int b0, const TcUnit* d_units, int nunits, int amax,
                        double thr, cudaStream_t st) {
  if (nunits <= 0) return;
  FMMLU_LAUNCH("xrr_fallback", st,
               k_ns_fallback<<<nunits, 512, (size_t)amax * sizeof(int), st>>>(L, b0, d_units, thr));
}

// ---------------------------------------------------------------------------
// root: block elimination of the dense n0 x n0 block (ld n0)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(512) k_root_diag(double2* A, int64_t n0, int i0, int r,
                                                   int* status) {
  __shared__ int ipiv[256];
  gauss_jordan(A + i0 + i0 * n0, r, n0, ipiv, status);
}

__global__ void __launch_bounds__(256) k_root_w(double2* A, int64_t n0, int i0, int r,
                                                double2* W) {
  int later = (int)(n0 - i0 - r);
  int tm, tn;
  if (!tile_of(later, r, tm, tn)) return;
  GemmArgs g{later, r, r, A + (i0 + r) + i0 * n0, n0, A + i0 + i0 * n0, n0};
  EpiStore e{W, later};
  gemm_tile<false, false>(g, tm, tn, e);
}

__global__ void __launch_bounds__(256) k_root_schur(double2* A, int64_t n0, int i0, int r,
                                                    const double2* W) {
  int later = (int)(n0 - i0 - r);
  int tm, tn;
  if (!tile_of(later, later, tm, tn)) return;
  int i1 = i0 + r;
  GemmArgs g{later, later, r, W, later, A + i0 + i1 * n0, n0};
  EpiSub e{A + i1 + i1 * n0, n0};
  gemm_tile<false, false>(g, tm, tn, e);
}

void launch_root_diag(double2* A, int n0, int i0, int r, int* status, cudaStream_t st) {
  FMMLU_LAUNCH("root_diag", st, k_root_diag<<<1, 512, 0, st>>>(A, n0, i0, r, status));
}

cudaError_t launch_root_factor(double2* A, int n0, int nb, double2* work, int* status,
                               cudaStream_t st, bool tensor_cores) {
  if (tensor_cores) return launch_root_factor_tc(A, n0, nb, work, status, st);
  for (int i0 = 0; i0 < n0; i0 += nb) {
    int r = std::min(nb, n0 - i0);
    FMMLU_LAUNCH("root_diag", st, k_root_diag<<<1, 512, 0, st>>>(A, n0, i0, r, status));
    int later = n0 - i0 - r;
    if (later > 0) {
      FMMLU_LAUNCH("root_w", st, k_root_w<<<tiles(later, r), 256, 0, st>>>(A, n0, i0, r, work));
      FMMLU_LAUNCH("root_schur", st,
                   k_root_schur<<<tiles(later, later), 256, 0, st>>>(A, n0, i0, r, work));
    }
  }
  return cudaGetLastError();
}

}  // namespace fmmlu
