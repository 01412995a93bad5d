// Application of the stored factors (Sec. 4.2, factored form of A^{-1}).
//
// Per eliminated box (idx = [R | S | N], C = S u N):
//   forward  (elimination order):  b_R -= T^T b_S; z = X_RR^{-1} b_R;
//                                  b_C -= X_CR z;  b_R = z
//   backward (reverse order):      x_R -= X_RR^{-1} (X_RC x_C); x_S -= T x_R
// Adjoint (A^{-H}):
//   forward:   b_R -= T^H b_S; z = X_RR^{-H} b_R; b_C -= X_RC^H z; b_R = z
//   backward:  x_R -= X_RR^{-H} (X_CR^H x_C);      x_S -= conj(T) x_R
// Boxes of one colour touch disjoint DOF sets (their closed neighbourhoods
// are disjoint), so one launch per colour is race free.
// Root: blocks D_i of the dense remainder, eliminated in order:
//   forward  z_i = D_i^{-1} b_i; b_later -= A[later, i] z_i
//   backward x_i = z_i - D_i^{-1} A[i, later] x_later
// (adjoint: the same with D_i^{-H}, A[i,later]^H, A[later,i]^H roles swapped).
#include "device_common.cuh"

namespace fmmlu {

__global__ void k_gather_vec(const double2* __restrict__ b, const int* __restrict__ perm,
                             int64_t n, double2* __restrict__ v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < n) v[c * n + i] = b[c * n + perm[i]];
}
__global__ void k_scatter_vec(const double2* __restrict__ v, const int* __restrict__ perm,
                              int64_t n, double2* __restrict__ x) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < n) x[c * n + perm[i]] = v[c * n + i];
}
void launch_gather_vec(const double2* b, const int* perm, int64_t n, int nrhs, double2* v,
                       cudaStream_t st) {
  FMMLU_LAUNCH("gather_vec", st, k_gather_vec<<<dim3((unsigned)((n + 255) / 256), nrhs), 256, 0, st>>>(b, perm, n, v));
}
void launch_scatter_vec(const double2* v, const int* perm, int64_t n, int nrhs, double2* x,
                        cudaStream_t st) {
  FMMLU_LAUNCH("scatter_vec", st, k_scatter_vec<<<dim3((unsigned)((n + 255) / 256), nrhs), 256, 0, st>>>(v, perm, n, x));
}

// Box sweeps, three launches per colour and direction, every product split
// into row chunks so that one large box uses many SMs (GB300's fp64 rate per
// SM is ~4 GFLOP/s, so one CTA per box would be bound by a single SM):
//   forward:  k_sw_y  (R chunks)  b_R -= op(T)^T b_S
//             k_sw_z  (R chunks)  z = op(X_RR^{-1}) b_R  (into the box's scratch)
//             k_fwd_c (C chunks)  b_C -= op(X_CR) z; the first chunk stores b_R = z
//   backward: k_bwd_t (C chunks)  partial = op(X_RC) x_C
//             k_sw_xr (R chunks)  x_R -= op(X_RR^{-1}) sum(partials)
//             k_sw_xs (S chunks)  x_S -= op(T) x_R
// op() is the identity for A^{-1}; for A^{-H} the roles are (X_RC^H, X_CR^H,
// X_RR^{-H}, conj(T)).

constexpr int kRowChunk = 16;   // output rows per CTA of the R and S products

// out[k - k0] = sum_l op(M)(k, l) x[l] for k in [k0, k0 + kc), kc <= 16, with
// 256 threads and x in shared memory. kRows: element (k, l) at M[k + l ld]
// (a half-warp reads 16 consecutive k); else at M[l + k ld] (16 consecutive
// l). cj conjugates the matrix element.
template <bool kRows>
__device__ __forceinline__ void chunk_mv(const double2* __restrict__ M, int64_t ld, bool cj,
                                         const double2* x, int L, int k0, int kc, double2* red,
                                         double2* out) {
  const int t = threadIdx.x;
  double2 acc = mk(0.0, 0.0);
  if (kRows) {
    const int row = t & 15, g = t >> 4;
    if (row < kc) {
      const double2* Mr = M + (k0 + row);
      for (int l = g; l < L; l += 16) {
        const double2 m = Mr[(int64_t)l * ld];
        if (cj) cfma_cj(acc, m, x[l]); else cfma(acc, m, x[l]);
      }
    }
    red[t] = acc;
    __syncthreads();
    if (t < kRowChunk) {
      double2 sum = mk(0.0, 0.0);
      for (int q = 0; q < 16; ++q) sum = cadd(sum, red[q * 16 + t]);
      out[t] = sum;
    }
  } else {
    const int row = t >> 4, ln = t & 15;
    if (row < kc) {
      const double2* Mc = M + (int64_t)(k0 + row) * ld;
      for (int l = ln; l < L; l += 16) {
        const double2 m = Mc[l];
        if (cj) cfma_cj(acc, m, x[l]); else cfma(acc, m, x[l]);
      }
    }
    for (int o = 8; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (ln == 0) out[row] = acc;
  }
  __syncthreads();
}

// forward: b_R[k] -= sum_i op(T)(i, k) b_S[i] for the chunk's rows k
__global__ void __launch_bounds__(256) k_sw_y(const SolveBox* __restrict__ boxes,
                                              const SweepItem* __restrict__ items, int i0,
                                              double2* __restrict__ v, int64_t n, int adjoint) {
  extern __shared__ double2 sh[];
  const SweepItem it = items[i0 + blockIdx.x];
  const SolveBox B = boxes[it.box];
  double2* vc = v + blockIdx.y * n;
  double2* red = sh;            // 256
  double2* out = sh + 256;      // 16
  double2* bS = sh + 272;       // s
  const int* Ridx = B.idx;
  const int* Sidx = B.idx + B.r;
  for (int i = threadIdx.x; i < B.s; i += blockDim.x) bS[i] = vc[Sidx[i]];
  __syncthreads();
  const int kc = it.c1 - it.c0;
  chunk_mv<false>(B.T, B.ldT, adjoint != 0, bS, B.s, it.c0, kc, red, out);
  if (threadIdx.x < kc) {
    const int dof = Ridx[it.c0 + threadIdx.x];
    vc[dof] = csub(vc[dof], out[threadIdx.x]);
  }
}

// forward: z = op(X_RR^{-1}) b_R for the chunk's rows, into the box's scratch
__global__ void __launch_bounds__(256) k_sw_z(const SolveBox* __restrict__ boxes,
                                              const SweepItem* __restrict__ items, int i0,
                                              const double2* __restrict__ v, int64_t n,
                                              double2* __restrict__ zbuf, int64_t zstride,
                                              int adjoint) {
  extern __shared__ double2 sh[];
  const SweepItem it = items[i0 + blockIdx.x];
  const SolveBox B = boxes[it.box];
  const double2* vc = v + blockIdx.y * n;
  double2* red = sh;
  double2* out = sh + 256;
  double2* y = sh + 272;        // r
  for (int k = threadIdx.x; k < B.r; k += blockDim.x) y[k] = vc[B.idx[k]];
  __syncthreads();
  const int kc = it.c1 - it.c0;
  if (!adjoint) chunk_mv<true>(B.Xinv, B.ldX, false, y, B.r, it.c0, kc, red, out);
  else chunk_mv<false>(B.Xinv, B.ldX, true, y, B.r, it.c0, kc, red, out);
  if (threadIdx.x < kc) zbuf[blockIdx.y * zstride + B.zoff + it.c0 + threadIdx.x] = out[threadIdx.x];
}

// backward: x_R[k] -= sum_l op(X_RR^{-1})(k, l) t[l], t = sum of the partials
__global__ void __launch_bounds__(256) k_sw_xr(const SolveBox* __restrict__ boxes,
                                               const SweepItem* __restrict__ items, int i0,
                                               double2* __restrict__ v, int64_t n,
                                               const double2* __restrict__ partial,
                                               int64_t pstride, int adjoint) {
  extern __shared__ double2 sh[];
  const SweepItem it = items[i0 + blockIdx.x];
  const SolveBox B = boxes[it.box];
  double2* vc = v + blockIdx.y * n;
  const double2* pc = partial + blockIdx.y * pstride;
  double2* red = sh;
  double2* out = sh + 256;
  double2* tt = sh + 272;       // r
  for (int k = threadIdx.x; k < B.r; k += blockDim.x) {
    double2 acc = mk(0.0, 0.0);
    for (int q = B.item_beg; q < B.item_beg + B.item_cnt; ++q) acc = cadd(acc, pc[items[q].part + k]);
    tt[k] = acc;
  }
  __syncthreads();
  const int kc = it.c1 - it.c0;
  if (!adjoint) chunk_mv<true>(B.Xinv, B.ldX, false, tt, B.r, it.c0, kc, red, out);
  else chunk_mv<false>(B.Xinv, B.ldX, true, tt, B.r, it.c0, kc, red, out);
  if (threadIdx.x < kc) {
    const int dof = B.idx[it.c0 + threadIdx.x];
    vc[dof] = csub(vc[dof], out[threadIdx.x]);
  }
}

// backward: x_S[i] -= sum_k op(T)(i, k) x_R[k] for the chunk's rows i
__global__ void __launch_bounds__(256) k_sw_xs(const SolveBox* __restrict__ boxes,
                                               const SweepItem* __restrict__ items, int i0,
                                               double2* __restrict__ v, int64_t n, int adjoint) {
  extern __shared__ double2 sh[];
  const SweepItem it = items[i0 + blockIdx.x];
  const SolveBox B = boxes[it.box];
  double2* vc = v + blockIdx.y * n;
  double2* red = sh;
  double2* out = sh + 256;
  double2* xr = sh + 272;       // r
  for (int k = threadIdx.x; k < B.r; k += blockDim.x) xr[k] = vc[B.idx[k]];
  __syncthreads();
  const int kc = it.c1 - it.c0;
  chunk_mv<true>(B.T, B.ldT, adjoint != 0, xr, B.r, it.c0, kc, red, out);
  if (threadIdx.x < kc) {
    const int dof = B.idx[B.r + it.c0 + threadIdx.x];
    vc[dof] = csub(vc[dof], out[threadIdx.x]);
  }
}

__global__ void __launch_bounds__(256) k_fwd_c(const SolveBox* __restrict__ boxes,
                                               const SweepItem* __restrict__ items, int i0,
                                               double2* __restrict__ v, int64_t n,
                                               const double2* __restrict__ zbuf, int64_t zstride,
                                               int adjoint) {
  extern __shared__ double2 z[];
  const SweepItem it = items[i0 + blockIdx.x];
  const SolveBox B = boxes[it.box];
  const int r = B.r;
  double2* vc = v + blockIdx.y * n;
  const double2* zc = zbuf + blockIdx.y * zstride + B.zoff;
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    z[k] = zc[k];
    if (it.c0 == 0) vc[B.idx[k]] = z[k];   // b_R = z, once per box
  }
  __syncthreads();
  const int* Cidx = B.idx + r;
  for (int i = it.c0 + threadIdx.x; i < it.c1; i += blockDim.x) {
    double2 acc = mk(0.0, 0.0);
    if (!adjoint)
      for (int k = 0; k < r; ++k) cfma(acc, B.XCR[i + (int64_t)k * B.ldL], z[k]);
    else
      for (int k = 0; k < r; ++k) cfma_cj(acc, B.XRC[k + (int64_t)i * B.ldU], z[k]);
    int dof = Cidx[i];
    vc[dof] = csub(vc[dof], acc);
  }
}

__global__ void __launch_bounds__(256) k_bwd_t(const SolveBox* __restrict__ boxes,
                                               const SweepItem* __restrict__ items, int i0,
                                               const double2* __restrict__ v, int64_t n,
                                               double2* __restrict__ partial, int64_t pstride,
                                               int adjoint) {
  extern __shared__ double2 sh[];
  const SweepItem it = items[i0 + blockIdx.x];
  const SolveBox B = boxes[it.box];
  const int r = B.r;
  const double2* vc = v + blockIdx.y * n;
  const int w = it.c1 - it.c0;
  double2* u = sh;            // chunk values of x_C
  double2* red = sh + w;      // 256
  const int* Cidx = B.idx + r;
  for (int j = threadIdx.x; j < w; j += blockDim.x) u[j] = vc[Cidx[it.c0 + j]];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double2* out = partial + blockIdx.y * pstride + it.part;
  for (int kb = 0; kb < r; kb += 32) {
    int k = kb + lane;
    double2 acc = mk(0.0, 0.0);
    if (k < r) {
      if (!adjoint)
        for (int j = warp; j < w; j += nw)
          cfma(acc, B.XRC[k + (int64_t)(it.c0 + j) * B.ldU], u[j]);
      else
        for (int j = warp; j < w; j += nw)
          cfma_cj(acc, B.XCR[(it.c0 + j) + (int64_t)k * B.ldL], u[j]);
    }
    red[warp * 32 + lane] = acc;
    __syncthreads();
    if (warp == 0 && k < r) {
      double2 t = mk(0.0, 0.0);
      for (int q = 0; q < nw; ++q) t = cadd(t, red[q * 32 + lane]);
      out[k] = t;
    }
    __syncthreads();
  }
}

static void set_smem_attr() {
  static bool done = false;
  if (done) return;
  for (const void* f : {(const void*)k_sw_y, (const void*)k_sw_z, (const void*)k_sw_xr,
                        (const void*)k_sw_xs, (const void*)k_fwd_c, (const void*)k_bwd_t})
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  done = true;
}

void launch_sweep(const SolveBox* boxes, const SweepItem* items, const SweepSeg& sg,
                  double2* v, int64_t n, int nrhs, bool backward, bool adjoint,
                  double2* partial, int64_t pstride, cudaStream_t st) {
  if (sg.nb <= 0) return;
  set_smem_attr();
  const int adj = adjoint ? 1 : 0;
  const size_t base = (size_t)(256 + kRowChunk) * sizeof(double2);
  if (!backward) {
    if (sg.smax > 0)
      FMMLU_LAUNCH("sweep_fwd", st,
                   k_sw_y<<<dim3(sg.nri, nrhs), 256, base + sg.smax * sizeof(double2), st>>>(
                       boxes, items, sg.ri0, v, n, adj));
    FMMLU_LAUNCH("sweep_fwd", st,
                 k_sw_z<<<dim3(sg.nri, nrhs), 256, base + sg.rmax * sizeof(double2), st>>>(
                     boxes, items, sg.ri0, v, n, partial, pstride, adj));
    FMMLU_LAUNCH("sweep_fwd_c", st,
                 k_fwd_c<<<dim3(sg.ni, nrhs), 256, (size_t)sg.rmax * sizeof(double2), st>>>(
                     boxes, items, sg.i0, v, n, partial, pstride, adj));
  } else {
    size_t sm1 = (size_t)(kSweepChunk + 256) * sizeof(double2);
    FMMLU_LAUNCH("sweep_bwd_t", st, k_bwd_t<<<dim3(sg.ni, nrhs), 256, sm1, st>>>(boxes, items, sg.i0, v, n,
                                                                               partial, pstride, adj));
    FMMLU_LAUNCH("sweep_bwd", st,
                 k_sw_xr<<<dim3(sg.nri, nrhs), 256, base + sg.rmax * sizeof(double2), st>>>(
                     boxes, items, sg.ri0, v, n, partial, pstride, adj));
    if (sg.nsi > 0)
      FMMLU_LAUNCH("sweep_bwd", st,
                   k_sw_xs<<<dim3(sg.nsi, nrhs), 256, base + sg.rmax * sizeof(double2), st>>>(
                       boxes, items, sg.si0, v, n, adj));
  }
}

// ---------------------------------------------------------------------------
// root

__global__ void k_root_gather(const double2* __restrict__ v, const int* __restrict__ dofs,
                              int n0, int64_t n, double2* __restrict__ vr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < n0) vr[(int64_t)c * n0 + i] = v[c * n + dofs[i]];
}
__global__ void k_root_scatter(const double2* __restrict__ vr, const int* __restrict__ dofs,
                               int n0, int64_t n, double2* __restrict__ v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < n0) v[c * n + dofs[i]] = vr[(int64_t)c * n0 + i];
}
void launch_root_gather(const double2* v, const int* dofs, int n0, int64_t n, int nrhs,
                        double2* vr, cudaStream_t st) {
  if (n0 <= 0) return;
  FMMLU_LAUNCH("root_gather", st, k_root_gather<<<dim3((n0 + 255) / 256, nrhs), 256, 0, st>>>(v, dofs, n0, n, vr));
}
void launch_root_scatter(const double2* vr, const int* dofs, int n0, int64_t n, int nrhs,
                         double2* v, cudaStream_t st) {
  if (n0 <= 0) return;
  FMMLU_LAUNCH("root_scatter", st, k_root_scatter<<<dim3((n0 + 255) / 256, nrhs), 256, 0, st>>>(vr, dofs, n0, n, v));
}

// forward step of block i: z_i = op(D_i^{-1}) b_i (every CTA recomputes it),
// then b_later -= op(A[later, i]) z_i on this CTA's rows; z_i stored in z.
constexpr int kRootRows = 256;
__global__ void __launch_bounds__(256) k_root_fwd(const double2* __restrict__ A, int64_t n0, int i0,
                                                  int r, double2* __restrict__ vr,
                                                  double2* __restrict__ z, int adjoint) {
  __shared__ double2 bi[256], zi[256];
  int c = blockIdx.y;
  double2* vc = vr + c * n0;
  double2* zc = z + c * n0;
  for (int k = threadIdx.x; k < r; k += blockDim.x) bi[k] = vc[i0 + k];
  __syncthreads();
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    double2 acc = mk(0.0, 0.0);
    for (int l = 0; l < r; ++l) {
      if (!adjoint) cfma(acc, A[(i0 + k) + (i0 + l) * n0], bi[l]);
      else cfma_cj(acc, A[(i0 + l) + (i0 + k) * n0], bi[l]);
    }
    zi[k] = acc;
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int k = threadIdx.x; k < r; k += blockDim.x) zc[i0 + k] = zi[k];
  int i1 = i0 + r;
  int row = i1 + blockIdx.x * kRootRows + threadIdx.x;
  if (row < n0) {
    double2 acc = mk(0.0, 0.0);
    for (int k = 0; k < r; ++k) {
      if (!adjoint) cfma(acc, A[row + (i0 + k) * n0], zi[k]);
      else cfma_cj(acc, A[(i0 + k) + row * n0], zi[k]);
    }
    vc[row] = csub(vc[row], acc);
  }
}

// backward, phase 1: partial[c][blk][k] = sum over this CTA's columns j of
// op(A[i, later])[k, j] x_j ; phase 2 reduces and applies x_i = z_i - D^{-1} t.
constexpr int kRootCols = 512;
__global__ void __launch_bounds__(256) k_root_bwd1(const double2* __restrict__ A, int64_t n0,
                                                   int i0, int r, const double2* __restrict__ x,
                                                   double2* __restrict__ partial, int nblk,
                                                   int adjoint) {
  __shared__ double2 red[256];
  int c = blockIdx.y;
  const double2* xc = x + c * n0;
  int i1 = i0 + r;
  int j0 = i1 + blockIdx.x * kRootCols;
  int j1 = min((int)n0, j0 + kRootCols);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int kb = 0; kb < r; kb += 32) {
    int k = kb + lane;
    double2 acc = mk(0.0, 0.0);
    if (k < r)
      for (int j = j0 + warp; j < j1; j += nw) {
        if (!adjoint) cfma(acc, A[(i0 + k) + (int64_t)j * n0], xc[j]);
        else cfma_cj(acc, A[j + (int64_t)(i0 + k) * n0], xc[j]);
      }
    red[warp * 32 + lane] = acc;
    __syncthreads();
    if (warp == 0 && k < r) {
      double2 s = mk(0.0, 0.0);
      for (int w = 0; w < nw; ++w) s = cadd(s, red[w * 32 + lane]);
      partial[((int64_t)c * nblk + blockIdx.x) * 256 + k] = s;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_root_bwd2(const double2* __restrict__ A, int64_t n0,
                                                   int i0, int r, double2* __restrict__ x,
                                                   const double2* __restrict__ z,
                                                   const double2* __restrict__ partial, int nblk,
                                                   int adjoint) {
  __shared__ double2 t[256];
  int c = blockIdx.x;
  double2* xc = x + c * n0;
  const double2* zc = z + c * n0;
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    double2 s = mk(0.0, 0.0);
    for (int p = 0; p < nblk; ++p) s = cadd(s, partial[((int64_t)c * nblk + p) * 256 + k]);
    t[k] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    double2 acc = mk(0.0, 0.0);
    for (int l = 0; l < r; ++l) {
      if (!adjoint) cfma(acc, A[(i0 + k) + (i0 + l) * n0], t[l]);
      else cfma_cj(acc, A[(i0 + l) + (i0 + k) * n0], t[l]);
    }
    xc[i0 + k] = csub(zc[i0 + k], acc);
  }
}

void launch_root_solve(const double2* A, int n0, int nb, double2* vr, double2* z,
                       double2* partial, int nrhs, bool adjoint, cudaStream_t st) {
  if (n0 <= 0) return;
  int adj = adjoint ? 1 : 0;
  for (int i0 = 0; i0 < n0; i0 += nb) {
    int r = std::min(nb, n0 - i0);
    int later = n0 - i0 - r;
    int nblk = std::max(1, (later + kRootRows - 1) / kRootRows);
    FMMLU_LAUNCH("root_fwd", st, k_root_fwd<<<dim3(nblk, nrhs), 256, 0, st>>>(A, n0, i0, r, vr, z, adj));
  }
  // backward: x := z, then blocks from last to first
  int nbl = (n0 + nb - 1) / nb;
  for (int bi = nbl - 1; bi >= 0; --bi) {
    int i0 = bi * nb;
    int r = std::min(nb, n0 - i0);
    int later = n0 - i0 - r;
    if (later > 0) {
      int nblk = (later + kRootCols - 1) / kRootCols;
      FMMLU_LAUNCH("root_bwd1", st, k_root_bwd1<<<dim3(nblk, nrhs), 256, 0, st>>>(
                                        A, n0, i0, r, vr, partial, nblk, adj));
      FMMLU_LAUNCH("root_bwd2", st, k_root_bwd2<<<nrhs, 256, 0, st>>>(A, n0, i0, r, vr, z, partial,
                                                                     nblk, adj));
    } else {
      FMMLU_LAUNCH("root_bwd2", st,
                   k_root_bwd2<<<nrhs, 256, 0, st>>>(A, n0, i0, r, vr, z, partial, 0, adj));
    }
  }
}

}  // namespace fmmlu
