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
#include <mutex>

#include "device_common.cuh"
#include "dfloat.cuh"

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
// SM is ~7 GFLOP/s, so one CTA per box would be bound by a single SM):
//   forward:  k_sw_y  (R chunks)  b_R -= op(T)^T b_S
//             k_sw_z  (R chunks)  z = op(X_RR^{-1}) b_R  (into the box's scratch)
//             k_fwd_c (C chunks)  b_C -= op(X_CR) z; the first chunk stores b_R = z
//   backward: k_bwd_t (C chunks)  partial = op(X_RC) x_C
//             k_sw_xr (R chunks)  x_R -= op(X_RR^{-1}) sum(partials)
//             k_sw_xs (S chunks)  x_S -= op(T) x_R
// op() is the identity for A^{-1}; for A^{-H} the roles are (X_RC^H, X_CR^H,
// X_RR^{-H}, conj(T)).
//
// Every product is a matrix-vector product of a column-major block with a
// vector staged in shared memory. At one right-hand side the block is read
// once, 16 B per 8 flops, so a CTA must keep many loads in flight: each thread
// issues four independent loads per step, and the threads are laid out so
// that a warp reads consecutive addresses (lanes over the contiguous index).

template <bool kCj>
__device__ __forceinline__ void cf(double2& acc, double2 a, double2 b) {
  if (kCj) cfma_cj(acc, a, b); else cfma(acc, a, b);
}

// store(o, y_o) with y_o = sum_{q < nq} op(M[o + q ld]) x[q], o < no: the
// output index is the contiguous one. 256 threads: consecutive threads take
// consecutive outputs (16 or 32 per tile); when fewer than 256 outputs are
// left, the remaining threads split q into interleaved groups whose sums meet
// in red (256 entries).
template <bool kCj, class Store>
__device__ __forceinline__ void mv_cols(const double2* __restrict__ M, int64_t ld,
                                        const double2* x, int no, int nq, double2* red,
                                        Store store) {
  const int t = threadIdx.x;
  const int ot = no <= 16 ? 16 : 32;
  int span = ot;
  while (span < no && span < 256) span <<= 1;
  const int qg = 256 / span;
  const int oi = t % span, g = t / span;
  for (int ob = 0; ob < no; ob += span) {
    const int o = ob + oi;
    double2 a0 = mk(0.0, 0.0), a1 = mk(0.0, 0.0);
    if (o < no) {
      const double2* Mo = M + o;
      int q = g;
      for (; q + 3 * qg < nq; q += 4 * qg) {
        const double2 m0 = Mo[(int64_t)q * ld];
        const double2 m1 = Mo[(int64_t)(q + qg) * ld];
        const double2 m2 = Mo[(int64_t)(q + 2 * qg) * ld];
        const double2 m3 = Mo[(int64_t)(q + 3 * qg) * ld];
        cf<kCj>(a0, m0, x[q]);
        cf<kCj>(a1, m1, x[q + qg]);
        cf<kCj>(a0, m2, x[q + 2 * qg]);
        cf<kCj>(a1, m3, x[q + 3 * qg]);
      }
      for (; q < nq; q += qg) cf<kCj>(a0, Mo[(int64_t)q * ld], x[q]);
    }
    const double2 acc = cadd(a0, a1);
    if (qg == 1) {
      if (o < no) store(o, acc);
    } else {
      red[t] = acc;
      __syncthreads();
      if (g == 0 && o < no) {
        double2 s = acc;
        for (int gg = 1; gg < qg; ++gg) s = cadd(s, red[gg * span + oi]);
        store(o, s);
      }
      __syncthreads();
    }
  }
}

// store(o, y_o) with y_o = sum_{q < nq} op(M[q + o ld]) x[q], o < no: every
// output is a dot product along a contiguous column. A group of 4 to 32 lanes
// per output, sized so that every lane takes at least four terms (the
// shuffle reduction inside the group costs fp64 adds of its own).
template <bool kCj, class Store>
__device__ __forceinline__ void mv_dots(const double2* __restrict__ M, int64_t ld,
                                        const double2* x, int no, int nq, Store store) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int sw = nq >= 128 ? 32 : (nq >= 64 ? 16 : (nq >= 32 ? 8 : 4));
  const int per = 32 / sw;
  const int sl = lane % sw, sub = lane / sw;
  for (int ob = w * per; ob < no; ob += nw * per) {
    const int o = ob + sub;
    double2 a0 = mk(0.0, 0.0), a1 = mk(0.0, 0.0);
    if (o < no) {
      const double2* Mo = M + (int64_t)o * ld;
      int q = sl;
      for (; q + 3 * sw < nq; q += 4 * sw) {
        const double2 m0 = Mo[q], m1 = Mo[q + sw], m2 = Mo[q + 2 * sw], m3 = Mo[q + 3 * sw];
        cf<kCj>(a0, m0, x[q]);
        cf<kCj>(a1, m1, x[q + sw]);
        cf<kCj>(a0, m2, x[q + 2 * sw]);
        cf<kCj>(a1, m3, x[q + 3 * sw]);
      }
      for (; q < nq; q += sw) cf<kCj>(a0, Mo[q], x[q]);
    }
    double2 acc = cadd(a0, a1);
    for (int off = sw >> 1; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (sl == 0 && o < no) store(o, acc);
  }
}

// ---------------------------------------------------------------------------
// Box sweeps in double-float arithmetic (dfloat.cuh), a group of NR
// right-hand sides per CTA (blockIdx.y = group): every block entry is read
// from HBM once per group and split into two fp32 numbers by integer
// operations, then applied to the NR right-hand sides staged in shared
// memory (complex double-float, X[cc * xs + q]). The vectors stay fp64; each
// result is rounded to fp64 once, where it is subtracted or stored.

// y[o][cc] = sum_{q < nq} op(M[o + q ld]) X[cc][q], o < no: the output index
// is the contiguous one. 256 threads: consecutive threads take consecutive
// outputs (16 or 32 per tile); when fewer than 256 outputs are left, the
// remaining threads split q into interleaved groups whose sums meet in red
// (256 entries per right-hand side, summed in a fixed group order).
// store(o, cc, y) receives the result of output o for right-hand side cc.
template <int NR, bool kCj, class Store>
__device__ __forceinline__ void mvr_cols(const double2* __restrict__ M, int64_t ld,
                                         const float4* X, int xs, int no, int nq, float4* red,
                                         Store store) {
  const int t = threadIdx.x;
  const int ot = no <= 16 ? 16 : 32;
  int span = ot;
  while (span < no && span < 256) span <<= 1;
  const int qg = 256 / span;
  const int oi = t % span, g = t / span;
  for (int ob = 0; ob < no; ob += span) {
    const int o = ob + oi;
    DF ar[NR], ai[NR];
#pragma unroll
    for (int cc = 0; cc < NR; ++cc) ar[cc] = ai[cc] = DF{0.f, 0.f};
    auto apply = [&](double2 m, int q) {
      const DF mr = df_split_bits(m.x), mi = df_split_bits(m.y);
#pragma unroll
      for (int cc = 0; cc < NR; ++cc) cdf_mac<kCj>(ar[cc], ai[cc], mr, mi, X[cc * xs + q]);
    };
    if (o < no) {
      const double2* Mo = M + o;
      int q = g;
      for (; q + qg < nq; q += 2 * qg) {
        const double2 m0 = Mo[(int64_t)q * ld];
        const double2 m1 = Mo[(int64_t)(q + qg) * ld];
        apply(m0, q);
        apply(m1, q + qg);
      }
      if (q < nq) apply(Mo[(int64_t)q * ld], q);
    }
    if (qg == 1) {
      if (o < no)
#pragma unroll
        for (int cc = 0; cc < NR; ++cc) store(o, cc, make_double2(df_value(ar[cc]), df_value(ai[cc])));
    } else {
#pragma unroll
      for (int cc = 0; cc < NR; ++cc)
        red[cc * 256 + t] = make_float4(ar[cc].h, ar[cc].l, ai[cc].h, ai[cc].l);
      __syncthreads();
      if (g == 0 && o < no) {
#pragma unroll
        for (int cc = 0; cc < NR; ++cc) {
          DF sr = ar[cc], si = ai[cc];
          for (int gg = 1; gg < qg; ++gg) {
            const float4 w = red[cc * 256 + gg * span + oi];
            sr = df_add(sr, DF{w.x, w.y});
            si = df_add(si, DF{w.z, w.w});
          }
          store(o, cc, make_double2(df_value(sr), df_value(si)));
        }
      }
      __syncthreads();
    }
  }
}

// y[o][cc] = sum_{q < nq} op(M[q + o ld]) X[cc][q], o < no: every output is a
// dot product along a contiguous column, taken by a group of 4 to 32 lanes
// and summed across the group with shuffles. The group is as small as still
// fills the CTA's 256 threads (each halving saves a shuffle round for all NR
// right-hand sides) and at most a quarter of nq (four terms per lane).
template <int NR, bool kCj, class Store>
__device__ __forceinline__ void mvr_dots(const double2* __restrict__ M, int64_t ld,
                                         const float4* X, int xs, int no, int nq, Store store) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int sw = 32;
  while (sw > 4 && (sw / 2) * no >= (int)blockDim.x) sw >>= 1;
  while (sw > 4 && nq < 4 * sw) sw >>= 1;
  const int per = 32 / sw;
  const int sl = lane % sw, sub = lane / sw;
  for (int ob = w * per; ob < no; ob += nw * per) {
    const int o = ob + sub;
    DF ar[NR], ai[NR];
#pragma unroll
    for (int cc = 0; cc < NR; ++cc) ar[cc] = ai[cc] = DF{0.f, 0.f};
    auto apply = [&](double2 m, int q) {
      const DF mr = df_split_bits(m.x), mi = df_split_bits(m.y);
#pragma unroll
      for (int cc = 0; cc < NR; ++cc) cdf_mac<kCj>(ar[cc], ai[cc], mr, mi, X[cc * xs + q]);
    };
    if (o < no) {
      const double2* Mo = M + (int64_t)o * ld;
      int q = sl;
      for (; q + sw < nq; q += 2 * sw) {
        const double2 m0 = Mo[q], m1 = Mo[q + sw];
        apply(m0, q);
        apply(m1, q + sw);
      }
      if (q < nq) apply(Mo[q], q);
    }
#pragma unroll
    for (int cc = 0; cc < NR; ++cc) {
      const DF sr = df_group_sum(ar[cc], sw), si = df_group_sum(ai[cc], sw);
      if (sl == 0 && o < no) store(o, cc, make_double2(df_value(sr), df_value(si)));
    }
  }
}

// X[cc][k] = split(value(cc, k)) for k < cnt and the group's right-hand
// sides (zeros past nrhs)
template <int NR, class Load>
__device__ __forceinline__ void stage_rhs(float4* X, int cnt, int cb, int nrhs, Load load) {
  for (int e = threadIdx.x; e < NR * cnt; e += blockDim.x) {
    const int cc = e / cnt, k = e - cc * cnt;
    X[e] = cb + cc < nrhs ? cdf_split_bits(load(cb + cc, k)) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// v[cb + cc][dof] -= y (a right-hand side of the group)
__device__ __forceinline__ void sub_rhs(double2* v, int64_t n, int cb, int cc, int nrhs, int dof,
                                        double2 y) {
  if (cb + cc >= nrhs) return;
  double2* p = v + (int64_t)(cb + cc) * n + dof;
  *p = csub(*p, y);
}

// forward: b_R[k] -= sum_i op(T)(i, k) b_S[i] for the chunk's rows k
template <int NR>
__global__ void __launch_bounds__(256, 4) k_sw_y(const SolveBox* __restrict__ boxes,
                                              const SweepItem* __restrict__ items, int i0,
                                              double2* __restrict__ v, int64_t n, int nrhs,
                                              int adjoint) {
  extern __shared__ float4 shf[];
  const SweepItem it = items[i0 + blockIdx.x];
  const SolveBox B = boxes[it.box];
  const int cb = blockIdx.y * NR;
  float4* X = shf;   // NR x s
  const int* Sidx = B.idx + B.r;
  stage_rhs<NR>(X, B.s, cb, nrhs, [&](int c, int i) { return v[(int64_t)c * n + Sidx[i]]; });
  __syncthreads();
  const int kc = it.c1 - it.c0;
  const int* Ridx = B.idx + it.c0;
  auto st = [=](int o, int cc, double2 y) { sub_rhs(v, n, cb, cc, nrhs, Ridx[o], y); };
  const double2* M = B.T + (int64_t)it.c0 * B.ldT;
  if (adjoint) mvr_dots<NR, true>(M, B.ldT, X, B.s, kc, B.s, st);
  else mvr_dots<NR, false>(M, B.ldT, X, B.s, kc, B.s, st);
}

// z_k = op(X_RR^{-1})(k, :) y for the chunk's rows k; store(k - c0, cc, z_k)
template <int NR, class Store>
__device__ __forceinline__ void xinv_rows(const SolveBox& B, int c0, int kc, const float4* Y,
                                          float4* red, bool adjoint, Store store) {
  if (!adjoint) mvr_cols<NR, false>(B.Xinv + c0, B.ldX, Y, B.r, kc, B.r, red, store);
  else mvr_dots<NR, true>(B.Xinv + (int64_t)c0 * B.ldX, B.ldX, Y, B.r, kc, B.r, store);
}

// forward: z = op(X_RR^{-1}) b_R for the chunk's rows, into the box's scratch
template <int NR>
__global__ void __launch_bounds__(256, 4) k_sw_z(const SolveBox* __restrict__ boxes,
                                              const SweepItem* __restrict__ items, int i0,
                                              const double2* __restrict__ v, int64_t n,
                                              double2* __restrict__ zbuf, int64_t zstride,
                                              int nrhs, int adjoint) {
  extern __shared__ float4 shf[];
  const SweepItem it = items[i0 + blockIdx.x];
  const SolveBox B = boxes[it.box];
  const int cb = blockIdx.y * NR;
  float4* red = shf;            // NR x 256
  float4* Y = shf + NR * 256;   // NR x r
  stage_rhs<NR>(Y, B.r, cb, nrhs, [&](int c, int k) { return v[(int64_t)c * n + B.idx[k]]; });
  __syncthreads();
  double2* zo = zbuf + B.zoff + it.c0;
  xinv_rows<NR>(B, it.c0, it.c1 - it.c0, Y, red, adjoint != 0, [=](int o, int cc, double2 z) {
    if (cb + cc < nrhs) zo[(int64_t)(cb + cc) * zstride + o] = z;
  });
}

// backward: x_R[k] -= sum_l op(X_RR^{-1})(k, l) t[l], t = the summed partials
template <int NR>
__global__ void __launch_bounds__(256, 4) k_sw_xr(const SolveBox* __restrict__ boxes,
                                               const SweepItem* __restrict__ items, int i0,
                                               double2* __restrict__ v, int64_t n,
                                               const double2* __restrict__ partial,
                                               int64_t pstride, int nrhs, int adjoint) {
  extern __shared__ float4 shf[];
  const SweepItem it = items[i0 + blockIdx.x];
  const SolveBox B = boxes[it.box];
  const int cb = blockIdx.y * NR;
  float4* red = shf;            // NR x 256
  float4* Tt = shf + NR * 256;  // NR x r
  stage_rhs<NR>(Tt, B.r, cb, nrhs,
                [&](int c, int k) { return partial[(int64_t)c * pstride + B.toff + k]; });
  __syncthreads();
  const int* Ridx = B.idx + it.c0;
  xinv_rows<NR>(B, it.c0, it.c1 - it.c0, Tt, red, adjoint != 0, [=](int o, int cc, double2 y) {
    sub_rhs(v, n, cb, cc, nrhs, Ridx[o], y);
  });
}

// backward: x_S[i] -= sum_k op(T)(i, k) x_R[k] for the chunk's rows i
template <int NR>
__global__ void __launch_bounds__(256, 4) k_sw_xs(const SolveBox* __restrict__ boxes,
                                               const SweepItem* __restrict__ items, int i0,
                                               double2* __restrict__ v, int64_t n, int nrhs,
                                               int adjoint) {
  extern __shared__ float4 shf[];
  const SweepItem it = items[i0 + blockIdx.x];
  const SolveBox B = boxes[it.box];
  const int cb = blockIdx.y * NR;
  float4* red = shf;            // NR x 256
  float4* Xr = shf + NR * 256;  // NR x r
  stage_rhs<NR>(Xr, B.r, cb, nrhs, [&](int c, int k) { return v[(int64_t)c * n + B.idx[k]]; });
  __syncthreads();
  const int* Sidx = B.idx + B.r + it.c0;
  auto st = [=](int o, int cc, double2 y) { sub_rhs(v, n, cb, cc, nrhs, Sidx[o], y); };
  if (adjoint) mvr_cols<NR, true>(B.T + it.c0, B.ldT, Xr, B.r, it.c1 - it.c0, B.r, red, st);
  else mvr_cols<NR, false>(B.T + it.c0, B.ldT, Xr, B.r, it.c1 - it.c0, B.r, red, st);
}

// forward: b_C -= op(X_CR) z on the chunk's rows of C
template <int NR>
__global__ void __launch_bounds__(256, 4) k_fwd_c(const SolveBox* __restrict__ boxes,
                                               const SweepItem* __restrict__ items, int i0,
                                               double2* __restrict__ v, int64_t n,
                                               const double2* __restrict__ zbuf, int64_t zstride,
                                               int nrhs, int adjoint) {
  extern __shared__ float4 shf[];
  const SweepItem it = items[i0 + blockIdx.x];
  const SolveBox B = boxes[it.box];
  const int r = B.r;
  const int cb = blockIdx.y * NR;
  float4* red = shf;            // NR x 256
  float4* Z = shf + NR * 256;   // NR x r
  stage_rhs<NR>(Z, r, cb, nrhs, [&](int c, int k) {
    const double2 zv = zbuf[(int64_t)c * zstride + B.zoff + k];
    if (it.c0 == 0) v[(int64_t)c * n + B.idx[k]] = zv;   // b_R = z, once per box
    return zv;
  });
  __syncthreads();
  const int* Cidx = B.idx + r + it.c0;
  auto st = [=](int o, int cc, double2 y) { sub_rhs(v, n, cb, cc, nrhs, Cidx[o], y); };
  const int w = it.c1 - it.c0;
  if (!adjoint) mvr_cols<NR, false>(B.XCR + it.c0, B.ldL, Z, r, w, r, red, st);
  else mvr_dots<NR, true>(B.XRC + (int64_t)it.c0 * B.ldU, B.ldU, Z, r, w, r, st);
}

// backward: partial = op(X_RC)[:, chunk] x_C[chunk] (r values per chunk and
// right-hand side); the last chunk of a box to finish (one counter per box
// and right-hand-side group, reset by that CTA; no CTA waits) sums the box's
// partials in chunk order into its t slots
template <int NR>
__global__ void __launch_bounds__(256, 4) k_bwd_t(const SolveBox* __restrict__ boxes,
                                               const SweepItem* __restrict__ items, int i0,
                                               const double2* __restrict__ v, int64_t n,
                                               double2* __restrict__ partial, int64_t pstride,
                                               int* __restrict__ cnt, int nrhs, int adjoint) {
  __shared__ int last;
  extern __shared__ float4 shf[];
  const SweepItem it = items[i0 + blockIdx.x];
  const SolveBox B = boxes[it.box];
  const int r = B.r;
  const int cb = blockIdx.y * NR;
  const int w = it.c1 - it.c0;
  float4* red = shf;            // NR x 256
  float4* U = shf + NR * 256;   // NR x w: the chunk's values of x_C
  const int* Cidx = B.idx + r;
  stage_rhs<NR>(U, w, cb, nrhs,
                [&](int c, int j) { return v[(int64_t)c * n + Cidx[it.c0 + j]]; });
  __syncthreads();
  auto st = [=](int o, int cc, double2 y) {
    if (cb + cc < nrhs) partial[(int64_t)(cb + cc) * pstride + it.part + o] = y;
  };
  if (!adjoint) mvr_cols<NR, false>(B.XRC + (int64_t)it.c0 * B.ldU, B.ldU, U, w, r, w, red, st);
  else mvr_dots<NR, true>(B.XCR + it.c0, B.ldL, U, w, r, w, st);
  int* ctr = cnt + (int64_t)it.box * gridDim.y + blockIdx.y;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ctr, 1) == B.item_cnt - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // t[k] = sum_j partial_j[k]: threads over k (rp of them) and over
  // interleaved groups of j, four loads in flight each, groups summed in a
  // fixed order (the result does not depend on which CTA came last)
  double2* redd = reinterpret_cast<double2*>(red);
  const int nc = B.item_cnt, t = threadIdx.x;
  const int rp = r <= 32 ? 32 : (r <= 64 ? 64 : (r <= 128 ? 128 : 256));
  const int G = 256 / rp, g = t / rp;
  for (int cc = 0; cc < NR && cb + cc < nrhs; ++cc) {
    const double2* pb = partial + (int64_t)(cb + cc) * pstride + B.zoff;
    double2* tb = partial + (int64_t)(cb + cc) * pstride + B.toff;
    for (int kb = 0; kb < r; kb += rp) {
      const int k = kb + t % rp;
      double2 a0 = mk(0.0, 0.0), a1 = mk(0.0, 0.0);
      if (k < r) {
        int j = g;
        for (; j + 3 * G < nc; j += 4 * G) {
          const double2 p0 = __ldcg(pb + (int64_t)j * r + k);
          const double2 p1 = __ldcg(pb + (int64_t)(j + G) * r + k);
          const double2 p2 = __ldcg(pb + (int64_t)(j + 2 * G) * r + k);
          const double2 p3 = __ldcg(pb + (int64_t)(j + 3 * G) * r + k);
          a0 = cadd(a0, cadd(p0, p2));
          a1 = cadd(a1, cadd(p1, p3));
        }
        for (; j < nc; j += G) a0 = cadd(a0, __ldcg(pb + (int64_t)j * r + k));
      }
      redd[t] = cadd(a0, a1);
      __syncthreads();
      if (g == 0 && k < r) {
        double2 sum = redd[t];
        for (int gg = 1; gg < G; ++gg) sum = cadd(sum, redd[gg * rp + t]);
        tb[k] = sum;
      }
      __syncthreads();
    }
  }
  if (t == 0) *ctr = 0;
}

// The dynamic shared-memory limit is a per-device attribute of each kernel:
// set it once per device (thread-safe), with that device current.
constexpr int kSmemAttrDevices = 64;
constexpr size_t kSweepSmemMax = 200 * 1024;
static std::once_flag g_smem_attr_once[kSmemAttrDevices];

template <int NR>
static void set_smem_attr_nr() {
  for (const void* f : {(const void*)k_sw_y<NR>, (const void*)k_sw_z<NR>,
                        (const void*)k_sw_xr<NR>, (const void*)k_sw_xs<NR>,
                        (const void*)k_fwd_c<NR>, (const void*)k_bwd_t<NR>})
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSweepSmemMax);
}

static void set_smem_attr() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kSmemAttrDevices) return;
  std::call_once(g_smem_attr_once[dev], [] {
    set_smem_attr_nr<1>();
    set_smem_attr_nr<2>();
    set_smem_attr_nr<4>();
    set_smem_attr_nr<8>();
  });
}

void prepare_solve_kernels() { set_smem_attr(); }

// b_R = z (forward sweep with the C product on the tensor cores)
__global__ void k_copy_z(const SolveBox* __restrict__ boxes, int b0, double2* __restrict__ v,
                         int64_t n, const double2* __restrict__ partial, int64_t pstride) {
  const SolveBox B = boxes[b0 + blockIdx.x];
  const int j = blockIdx.y;
  double2* vc = v + j * n;
  const double2* z = partial + j * pstride + B.zoff;
  for (int k = threadIdx.x; k < B.r; k += blockDim.x) vc[B.idx[k]] = z[k];
}

void launch_copy_z(const SolveBox* boxes, int b0, int nb, int rmax, double2* v, int64_t n,
                   int nrhs, const double2* partial, int64_t pstride, cudaStream_t st) {
  if (nb <= 0) return;
  const int th = rmax >= 256 ? 256 : rmax >= 64 ? 128 : 64;
  FMMLU_LAUNCH("sweep_fwd", st,
               k_copy_z<<<dim3(nb, nrhs), th, 0, st>>>(boxes, b0, v, n, partial, pstride));
}

template <int NR>
static void launch_sweep_nr(const SolveBox* boxes, const SweepItem* items, const SweepSeg& sg,
                            double2* v, int64_t n, int nrhs, bool backward, int adj,
                            double2* partial, int64_t pstride, cudaStream_t st, int* cnt,
                            bool skip_c) {
  const unsigned ng = (unsigned)((nrhs + NR - 1) / NR);
  const size_t red = (size_t)NR * 256 * sizeof(float4);
  const size_t smr = red + (size_t)NR * sg.rmax * sizeof(float4);
  if (!backward) {
    if (sg.smax > 0)
      FMMLU_LAUNCH("sweep_fwd", st,
                   k_sw_y<NR><<<dim3(sg.nri, ng), 256, (size_t)NR * sg.smax * sizeof(float4), st>>>(
                       boxes, items, sg.ri0, v, n, nrhs, adj));
    FMMLU_LAUNCH("sweep_fwd", st,
                 k_sw_z<NR><<<dim3(sg.nri, ng), 256, smr, st>>>(boxes, items, sg.ri0, v, n,
                                                                partial, pstride, nrhs, adj));
    if (!skip_c)
      FMMLU_LAUNCH("sweep_fwd_c", st,
                   k_fwd_c<NR><<<dim3(sg.ni, ng), 256, smr, st>>>(boxes, items, sg.i0, v, n,
                                                                  partial, pstride, nrhs, adj));
  } else {
    const size_t sm1 = red + (size_t)NR * sg.chunk * sizeof(float4);
    if (!skip_c)
      FMMLU_LAUNCH("sweep_bwd_t", st,
                   k_bwd_t<NR><<<dim3(sg.ni, ng), 256, sm1, st>>>(boxes, items, sg.i0, v, n,
                                                                    partial, pstride, cnt, nrhs,
                                                                    adj));
    FMMLU_LAUNCH("sweep_bwd", st,
                 k_sw_xr<NR><<<dim3(sg.nri, ng), 256, smr, st>>>(boxes, items, sg.ri0, v, n,
                                                                 partial, pstride, nrhs, adj));
    if (sg.nsi > 0)
      FMMLU_LAUNCH("sweep_bwd", st,
                   k_sw_xs<NR><<<dim3(sg.nsi, ng), 256, smr, st>>>(boxes, items, sg.si0, v, n,
                                                                   nrhs, adj));
  }
}

static int sweep_group_size(int nrhs, int qmax) {
  // the largest group (at most 8, at most the next power of two above nrhs)
  // whose staged right-hand sides and reduction buffer fit in shared memory
  int nr = 8;
  while (nr > 1 && (nr / 2 >= nrhs || (size_t)nr * (256 + qmax) * sizeof(float4) > kSweepSmemMax))
    nr >>= 1;
  return nr;
}

void launch_sweep(const SolveBox* boxes, const SweepItem* items, const SweepSeg& sg,
                  double2* v, int64_t n, int nrhs, bool backward, bool adjoint,
                  double2* partial, int64_t pstride, cudaStream_t st, int* cnt, bool skip_c) {
  if (sg.nb <= 0) return;
  set_smem_attr();
  const int adj = adjoint ? 1 : 0;
  const int nr = sweep_group_size(nrhs, std::max(std::max(sg.rmax, sg.smax), sg.chunk));
  switch (nr) {
    case 8: launch_sweep_nr<8>(boxes, items, sg, v, n, nrhs, backward, adj, partial, pstride, st, cnt, skip_c); break;
    case 4: launch_sweep_nr<4>(boxes, items, sg, v, n, nrhs, backward, adj, partial, pstride, st, cnt, skip_c); break;
    case 2: launch_sweep_nr<2>(boxes, items, sg, v, n, nrhs, backward, adj, partial, pstride, st, cnt, skip_c); break;
    default: launch_sweep_nr<1>(boxes, items, sg, v, n, nrhs, backward, adj, partial, pstride, st, cnt, skip_c); break;
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

// forward step of block i: z_i = op(D_i^{-1}) b_i (every CTA recomputes it
// from L2), then b_later -= op(A[later, i]) z_i on this CTA's kRootRows rows;
// z_i stored in z.
constexpr int kRootRows = 64;
constexpr int kRootCols = 128;
constexpr int kRootMaxBlock = 256;
__global__ void __launch_bounds__(256) k_root_fwd(const double2* __restrict__ A, int64_t n0, int i0,
                                                  int r, double2* __restrict__ vr,
                                                  double2* __restrict__ z, int adjoint) {
  __shared__ double2 bi[kRootMaxBlock], zi[kRootMaxBlock], red[256];
  const int c = blockIdx.y;
  double2* vc = vr + c * n0;
  double2* zc = z + c * n0;
  for (int k = threadIdx.x; k < r; k += blockDim.x) bi[k] = vc[i0 + k];
  __syncthreads();
  const double2* D = A + i0 + (int64_t)i0 * n0;
  double2* zip = zi;
  auto sz = [=](int o, double2 y) { zip[o] = y; };
  if (!adjoint) mv_cols<false>(D, n0, bi, r, r, red, sz);
  else mv_dots<true>(D, n0, bi, r, r, sz);
  __syncthreads();
  if (blockIdx.x == 0)
    for (int k = threadIdx.x; k < r; k += blockDim.x) zc[i0 + k] = zi[k];
  const int row0 = i0 + r + blockIdx.x * kRootRows;
  const int nrow = min(kRootRows, (int)n0 - row0);
  if (nrow <= 0) return;
  auto su = [=](int o, double2 y) { vc[row0 + o] = csub(vc[row0 + o], y); };
  if (!adjoint) mv_cols<false>(A + row0 + (int64_t)i0 * n0, n0, zi, nrow, r, red, su);
  else mv_dots<true>(A + i0 + (int64_t)row0 * n0, n0, zi, nrow, r, su);
}

// backward step of block i: every CTA forms partial = op(A[i, later]) x_later
// over its kRootCols columns; the last CTA to finish (one counter per
// right-hand side, reset by that CTA) sums the partials and applies
// x_i = z_i - op(D_i^{-1}) (sum). No CTA waits for another.
__global__ void __launch_bounds__(256) k_root_bwd(const double2* __restrict__ A, int64_t n0,
                                                  int i0, int r, double2* __restrict__ x,
                                                  const double2* __restrict__ z,
                                                  double2* __restrict__ partial, int pst,
                                                  int* __restrict__ cnt, int adjoint) {
  __shared__ double2 u[kRootCols], t[kRootMaxBlock], red[256];
  __shared__ int last;
  const int c = blockIdx.y, nblk = gridDim.x;
  double2* xc = x + c * n0;
  const double2* zc = z + c * n0;
  const int j0 = i0 + r + blockIdx.x * kRootCols;
  const int nj = max(0, min(kRootCols, (int)n0 - j0));
  for (int j = threadIdx.x; j < nj; j += blockDim.x) u[j] = xc[j0 + j];
  __syncthreads();
  double2* pc = partial + ((int64_t)c * nblk + blockIdx.x) * pst;
  auto sp = [=](int o, double2 y) { pc[o] = y; };
  if (nj > 0) {
    if (!adjoint) mv_cols<false>(A + i0 + (int64_t)j0 * n0, n0, u, r, nj, red, sp);
    else mv_dots<true>(A + j0 + (int64_t)i0 * n0, n0, u, r, nj, sp);
  } else {
    for (int k = threadIdx.x; k < r; k += blockDim.x) pc[k] = mk(0.0, 0.0);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&cnt[c], 1) == nblk - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    double2 s = mk(0.0, 0.0);
    for (int p = 0; p < nblk; ++p) s = cadd(s, __ldcg(&partial[((int64_t)c * nblk + p) * pst + k]));
    t[k] = s;
  }
  __syncthreads();
  const double2* D = A + i0 + (int64_t)i0 * n0;
  auto sx = [=](int o, double2 y) { xc[i0 + o] = csub(zc[i0 + o], y); };
  if (!adjoint) mv_cols<false>(D, n0, t, r, r, red, sx);
  else mv_dots<true>(D, n0, t, r, r, sx);
  if (threadIdx.x == 0) cnt[c] = 0;
}

size_t root_solve_scratch_bytes(int n0, int nb, int nrhs) {
  if (n0 <= 0) return 0;
  const size_t nblk = std::max(1, (n0 + kRootCols - 1) / kRootCols);
  const size_t part = ((size_t)nrhs * nblk * nb * sizeof(double2) + 255) & ~(size_t)255;
  return part + (((size_t)nrhs * sizeof(int) + 255) & ~(size_t)255);
}

cudaError_t launch_root_solve(const double2* A, int n0, int nb, double2* vr, double2* z,
                              void* scratch, int nrhs, bool adjoint, cudaStream_t st) {
  if (n0 <= 0) return cudaSuccess;
  if (nb < 1 || nb > kRootMaxBlock) return cudaErrorInvalidValue;
  const int adj = adjoint ? 1 : 0;
  const size_t nblk_max = std::max(1, (n0 + kRootCols - 1) / kRootCols);
  const size_t part_bytes = ((size_t)nrhs * nblk_max * nb * sizeof(double2) + 255) & ~(size_t)255;
  double2* partial = static_cast<double2*>(scratch);
  int* cnt = reinterpret_cast<int*>(static_cast<unsigned char*>(scratch) + part_bytes);
  cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)nrhs * sizeof(int), st);
  if (e != cudaSuccess) return e;
  for (int i0 = 0; i0 < n0; i0 += nb) {
    const int r = std::min(nb, n0 - i0);
    const int later = n0 - i0 - r;
    const int nblk = std::max(1, (later + kRootRows - 1) / kRootRows);
    FMMLU_LAUNCH("root_fwd", st, k_root_fwd<<<dim3(nblk, nrhs), 256, 0, st>>>(A, n0, i0, r, vr, z, adj));
  }
  // backward: blocks from last to first; x overwrites vr
  const int nbl = (n0 + nb - 1) / nb;
  for (int bi = nbl - 1; bi >= 0; --bi) {
    const int i0 = bi * nb;
    const int r = std::min(nb, n0 - i0);
    const int later = n0 - i0 - r;
    const int nblk = std::max(1, (later + kRootCols - 1) / kRootCols);
    FMMLU_LAUNCH("root_bwd", st, k_root_bwd<<<dim3(nblk, nrhs), 256, 0, st>>>(
                                     A, n0, i0, r, vr, z, partial, nb, cnt, adj));
  }
  return cudaGetLastError();
}

}  // namespace fmmlu
