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

// t[k] = sum_j op(M)[k, j] u[j] for k < rows, j < cols, where op(M)[k,j] =
// M[k + j ld] (conj = false) or conj(M[j + k ld]) (transposed-conjugated).
// Result in shared t[]; all threads of the block participate.
template <bool CONJT>
__device__ void block_matvec_red(const double2* __restrict__ M, int64_t ld, int rows, int cols,
                                 const double2* u_sh, double2* t, double2* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int kb = 0; kb < rows; kb += 32) {
    int k = kb + lane;
    double2 acc = mk(0.0, 0.0);
    if (k < rows) {
      for (int j = warp; j < cols; j += nw) {
        if (!CONJT) cfma(acc, M[k + j * ld], u_sh[j]);
        else cfma_cj(acc, M[j + (int64_t)k * ld], u_sh[j]);
      }
    }
    red[warp * 32 + lane] = acc;
    __syncthreads();
    if (warp == 0) {
      double2 s = mk(0.0, 0.0);
      for (int w = 0; w < nw; ++w) s = cadd(s, red[w * 32 + lane]);
      if (k < rows) t[k] = s;
    }
    __syncthreads();
  }
}

// Box sweep. Shared memory: bR, z (rmax each), u (rmax + s + n capped: we
// stage the gathered C-part in chunks through global reads instead).
__global__ void __launch_bounds__(256) k_sweep(const SolveBox* __restrict__ boxes, int b0,
                                               double2* __restrict__ v, int64_t n, int backward,
                                               int adjoint, int rmax) {
  extern __shared__ double2 sh[];
  const SolveBox B = boxes[b0 + blockIdx.x];
  const int r = B.r, s = B.s, nn = B.n;
  if (r == 0) return;
  const int c = blockIdx.y;
  double2* vc = v + c * n;
  double2* t1 = sh;              // rmax
  double2* t2 = sh + rmax;       // rmax
  double2* red = sh + 2 * rmax;  // 256
  double2* u = red + 256;        // staging for gathered vectors (rmax + chunk)
  const int* Ridx = B.idx;
  const int* Sidx = B.idx + r;
  const int* Cidx = B.idx + r;   // C = [S | N]
  const int tid = threadIdx.x;
  const int m = s + nn;
  if (!backward) {
    // t1 = b_R - op(T)^T b_S
    for (int k = tid; k < r; k += blockDim.x) {
      double2 acc = vc[Ridx[k]];
      for (int i = 0; i < s; ++i) {
        double2 tv = B.T[i + (int64_t)k * B.ldT];
        double2 bs = vc[Sidx[i]];
        if (!adjoint) acc = csub(acc, cmul(tv, bs));
        else acc = csub(acc, cmul(cconj(tv), bs));
      }
      t1[k] = acc;
    }
    __syncthreads();
    // t2 = Xinv t1  (or Xinv^H t1)
    for (int k = tid; k < r; k += blockDim.x) {
      double2 acc = mk(0.0, 0.0);
      for (int l = 0; l < r; ++l) {
        if (!adjoint) cfma(acc, B.Xinv[k + (int64_t)l * B.ldX], t1[l]);
        else cfma_cj(acc, B.Xinv[l + (int64_t)k * B.ldX], t1[l]);
      }
      t2[k] = acc;
    }
    __syncthreads();
    // b_C -= X_CR t2   (or X_RC^H t2)
    for (int i = tid; i < m; i += blockDim.x) {
      double2 acc = mk(0.0, 0.0);
      for (int k = 0; k < r; ++k) {
        if (!adjoint) cfma(acc, B.XCR[i + (int64_t)k * B.ldL], t2[k]);
        else cfma_cj(acc, B.XRC[k + (int64_t)i * B.ldU], t2[k]);
      }
      int dof = Cidx[i];
      vc[dof] = csub(vc[dof], acc);
    }
    for (int k = tid; k < r; k += blockDim.x) vc[Ridx[k]] = t2[k];
  } else {
    // t1 = op(X_RC) x_C, reduction over the m columns, staged in chunks
    for (int k = tid; k < r; k += blockDim.x) t1[k] = mk(0.0, 0.0);
    __syncthreads();
    const int chunk = 1024;
    for (int j0 = 0; j0 < m; j0 += chunk) {
      int jl = min(chunk, m - j0);
      for (int j = tid; j < jl; j += blockDim.x) u[j] = vc[Cidx[j0 + j]];
      __syncthreads();
      if (!adjoint)
        block_matvec_red<false>(B.XRC + (int64_t)j0 * B.ldU, B.ldU, r, jl, u, t2, red);
      else
        block_matvec_red<true>(B.XCR + j0, B.ldL, r, jl, u, t2, red);
      for (int k = tid; k < r; k += blockDim.x) t1[k] = cadd(t1[k], t2[k]);
      __syncthreads();
    }
    // x_R = b_R - op(Xinv) t1
    for (int k = tid; k < r; k += blockDim.x) {
      double2 acc = mk(0.0, 0.0);
      for (int l = 0; l < r; ++l) {
        if (!adjoint) cfma(acc, B.Xinv[k + (int64_t)l * B.ldX], t1[l]);
        else cfma_cj(acc, B.Xinv[l + (int64_t)k * B.ldX], t1[l]);
      }
      t2[k] = csub(vc[Ridx[k]], acc);
    }
    __syncthreads();
    for (int k = tid; k < r; k += blockDim.x) vc[Ridx[k]] = t2[k];
    // x_S -= op(T) x_R
    for (int i = tid; i < s; i += blockDim.x) {
      double2 acc = mk(0.0, 0.0);
      for (int k = 0; k < r; ++k) {
        double2 tv = B.T[i + (int64_t)k * B.ldT];
        if (!adjoint) cfma(acc, tv, t2[k]);
        else cfma(acc, cconj(tv), t2[k]);
      }
      vc[Sidx[i]] = csub(vc[Sidx[i]], acc);
    }
  }
}

void launch_sweep(const SolveBox* boxes, int b0, int nb, int rmax, double2* v, int64_t n,
                  int nrhs, bool backward, bool adjoint, cudaStream_t st) {
  if (nb <= 0 || rmax <= 0) return;
  size_t sm = (size_t)(2 * rmax + 256 + 1024) * sizeof(double2);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  FMMLU_LAUNCH(backward ? "sweep_bwd" : "sweep_fwd", st,
               k_sweep<<<dim3(nb, nrhs), 256, sm, st>>>(boxes, b0, v, n, backward ? 1 : 0,
                                                       adjoint ? 1 : 0, rmax));
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
