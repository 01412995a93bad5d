// Schur update Delta[C, C] -= W X_RC on the bf16 tensor cores, by an exact
// splitting of the complex128 operands (Ozaki-type scheme).
//
// Splitting. Row i of W is scaled by 2^-E_i (E_i = exponent of the row's
// largest real or imaginary part) so every scaled entry lies in (-1, 1); its
// base-256 digits d_0..d_6 (integers in [-255, 255], exact in bf16) satisfy
//   W_ik = 2^E_i * sum_p d_p 2^{-8(p+1)} + O(2^{E_i - 56}).
// Columns of X_RC get exponents F_j and digits e_q the same way. Then
//   (W X_RC)_ij = 2^{E_i + F_j} sum_{p+q<=6} 2^{-8(p+q+2)} sum_k d_p(ik) e_q(kj)
// up to a relative 2^-53-level truncation. Each inner sum over a block of at
// most 128 k, with the two real products that form one complex part, stays
// below 2 * 128 * 255^2 < 2^24, so the fp32 tensor-core accumulation of those
// integer products is exact. The exact block sums of all pairs with the same
// p + q (one power-of-two scale) are added as int32 (at most 7 (K/128) 2^24 <
// 2^31 for K <= 2048; longer K flushes early), converted to fp64 once per
// p + q, scaled and accumulated in fp64, then scaled by 2^{E_i + F_j} and
// subtracted from the fp64 Delta blocks: every product and partial sum is
// exact and every rounding is an fp64 addition.
#include <cuda_bf16.h>

#include <algorithm>

#include "device_common.cuh"

namespace fmmlu {

constexpr int kOzSlices = 7;
constexpr int kOzMinK = kOzInnerMin;   // smaller inner dimensions use the fp64 FMA kernels

using OzBox = OzBoxHost;

__device__ __forceinline__ int row_exponent(double m) {
  int e = 0;
  if (m > 0.0) frexp(m, &e);   // m < 2^e
  return e;
}

// v * 2^-e in (-1, 1): its first NS signed base-256 digits (each an integer
// in [-255, 255], exact in bf16). The scaled value times 2^(8 NS) is truncated
// to an integer U (one exact scaling and one conversion); digit p is byte
// NS - 1 - p of |U| with the sign of v -- the same digits as repeatedly
// scaling by 256 and truncating.
template <int NS>
__device__ __forceinline__ void split_digits_n(double v, int e, __nv_bfloat16* out,
                                               int64_t stride) {
  static_assert(NS >= 1 && NS <= 7, "at most 56 bits");
  const long long F = (long long)ldexp(v, 8 * NS - e);   // |F| < 2^(8 NS), toward 0
  const bool neg = F < 0;
  const unsigned long long U = (unsigned long long)(neg ? -F : F);
#pragma unroll
  for (int p = 0; p < NS; ++p) {
    int dgt = (int)((U >> (8 * (NS - 1 - p))) & 255ull);
    out[p * stride] = __int2bfloat16_rn(neg ? -dgt : dgt);
  }
}
__device__ __forceinline__ void split_digits(double v, int e, __nv_bfloat16* out,
                                             int64_t stride) {
  split_digits_n<kOzSlices>(v, e, out, stride);
}

// One CTA per (box, 32-row chunk) of W (rows) or of X_RC (columns).
__global__ void __launch_bounds__(256) k_oz_split(LevelDev L, int b0, const OzBox* __restrict__ oz,
                                                  __nv_bfloat16* slices, int* expo) {
  const int b = b0 + blockIdx.z;
  const BoxDesc d = L.desc[b];
  const BoxRun run = L.run[b];
  const int s = run.s, r = run.r, n = run.n;
  if (r < kOzMinK) return;
  const OzBox o = oz[blockIdx.z];
  const int m = s + n;
  const int mt = (m + 63) & ~63;
  const int kt = (r + 15) & ~15;
  const bool cols = blockIdx.y == 1;
  const int i0 = blockIdx.x * 32;
  if (i0 >= mt) return;
  const int64_t lw = d.a + d.nmax;
  const double2* W = L.Wbuf + d.W_off;                 // (m x r), ld lw
  const double2* X = L.arena + d.G1_off + s;           // X_RC(k, j) = X[k + j a]
  __nv_bfloat16* base = slices + (cols ? o.b_off : o.a_off);
  int* ex = expo + o.e_off + (cols ? o.mpad : 0);
  const int64_t pstride = 2 * (int64_t)o.mpad * o.kp;  // one slice, both parts
  const int64_t partstride = (int64_t)o.mpad * o.kp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int rr = warp; rr < 32; rr += 8) {
    const int i = i0 + rr;
    if (i >= mt) break;
    double mx = 0.0;
    if (i < m)
      for (int k = lane; k < r; k += 32) {
        double2 v = cols ? X[k + (int64_t)i * d.a] : W[i + (int64_t)k * lw];
        mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
      }
    for (int o2 = 16; o2 > 0; o2 >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o2));
    const int e = row_exponent(mx);
    if (lane == 0) ex[i] = e;
    for (int k = lane; k < kt; k += 32) {
      double2 v = make_double2(0.0, 0.0);
      if (i < m && k < r) v = cols ? X[k + (int64_t)i * d.a] : W[i + (int64_t)k * lw];
      __nv_bfloat16* dst = base + (int64_t)i * o.kp + k;
      split_digits(v.x, e, dst, pstride);
      split_digits(v.y, e, dst + partstride, pstride);
    }
  }
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory staging of one slice block: 64 rows x 128 k of bf16 for the
// real and the imaginary part, rows padded to 136 elements (272 B) so that the
// 8 row addresses of an ldmatrix hit distinct bank groups.
constexpr int kOzKB = 128;
constexpr int kOzLd = kOzKB + 8;
constexpr int kOzStage = 2 * 64 * kOzLd;    // bf16 elements per staged block

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// stage rows [r0, r0+64), k in [kb, kb + klen) of one slice (both parts)
__device__ __forceinline__ void stage_block(__nv_bfloat16* dst, const __nv_bfloat16* src,
                                            int64_t partstride, int kp, int r0, int kb, int klen) {
  const int chunks = klen / 8;                 // 16-byte chunks per row
  const int total = 2 * 64 * chunks;
  for (int c = threadIdx.x; c < total; c += blockDim.x) {
    int part = c / (64 * chunks);
    int rem = c - part * 64 * chunks;
    int row = rem / chunks, ch = rem - row * chunks;
    const __nv_bfloat16* g = src + part * partstride + (int64_t)(r0 + row) * kp + kb + ch * 8;
    cp_async16(dst + part * 64 * kOzLd + row * kOzLd + ch * 8, g);
  }
}

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const __nv_bfloat16* p) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// The digit-pair products of one 64 x 64 output tile: for every scale
// d = p + q <= DMAX (digits p, q < NS), stage A_p and B_q blocks (cp.async,
// double-buffered), multiply on the tensor cores (exact fp32 block sums), add
// the pairs of equal scale as int32 and accumulate each scale once in fp64.
// acc receives the tile of sum 2^{-8(p+q+2)} (op(A_p) B_q) (before the row and
// column exponents), op = conjugation when ConjA.
template <int NS, int DMAX, bool ConjA>
__device__ __forceinline__ void oz_tile_acc(__nv_bfloat16* sm, const __nv_bfloat16* Asl,
                                            const __nv_bfloat16* Bsl, int64_t partstride, int kp,
                                            int i0, int j0, int kt, double (&acc)[4][4][2]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wr = (warp & 3) * 16;
  const int wc = (warp >> 2) * 32;
  const int64_t pstride = 2 * partstride;
  // ldmatrix row addresses (element offsets inside a staged part)
  const int mi = lane >> 3, ri = lane & 7;
  const int a_off = (wr + ri + (mi & 1) * 8) * kOzLd + (mi >> 1) * 8;
  // B: matrices (n 0-7,k 0-7), (n 0-7,k 8-15), (n 8-15,k 0-7), (n 8-15,k 8-15)
  const int b_off = (wc + ri + (mi >> 1) * 8) * kOzLd + (mi & 1) * 8;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[u][e][0] = acc[u][e][1] = 0.0;
  // stages: (d, kb, p) with q = d - p; A_p and B_q blocks double-buffered
  const int nkb = (kt + kOzKB - 1) / kOzKB;
  auto plo = [](int d) { return d > NS - 1 ? d - (NS - 1) : 0; };
  auto phi = [](int d) { return d < NS - 1 ? d : NS - 1; };
  auto stage = [&](int d, int kb_i, int p, int buf) {
    const int kb = kb_i * kOzKB, klen = min(kOzKB, kt - kb);
    __nv_bfloat16* dA = sm + buf * 2 * kOzStage;
    stage_block(dA, Asl + p * pstride, partstride, kp, i0, kb, klen);
    stage_block(dA + kOzStage, Bsl + (d - p) * pstride, partstride, kp, j0, kb, klen);
    cp_async_commit();
  };
  int buf = 0;
  __syncthreads();
  stage(0, 0, 0, 0);
  for (int d = 0; d <= DMAX; ++d) {
    int G[4][4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int e = 0; e < 4; ++e) G[u][e][0] = G[u][e][1] = 0;
    int gcount = 0;
    const double scale = ldexp(1.0, -8 * (d + 2));
    for (int kb_i = 0; kb_i < nkb; ++kb_i) {
      for (int p = plo(d); p <= phi(d); ++p) {
        cp_async_wait_all();
        __syncthreads();
        // prefetch the next stage into the other buffer
        int nd = d, nk = kb_i, np = p + 1;
        if (np > phi(nd)) { np = plo(nd); ++nk; }
        if (nk >= nkb) { nk = 0; ++nd; np = plo(nd); }
        if (nd <= DMAX) stage(nd, nk, np, buf ^ 1);
        const __nv_bfloat16* sA = sm + buf * 2 * kOzStage;
        const __nv_bfloat16* sB = sA + kOzStage;
        const int klen = min(kOzKB, kt - kb_i * kOzKB);
        float cr[4][4], ci[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int e = 0; e < 4; ++e) cr[u][e] = ci[u][e] = 0.f;
        for (int k0 = 0; k0 < klen; k0 += 16) {
          uint32_t ar[4], ai[4], an[4];
          ldsm_x4(ar, sA + a_off + k0);
          ldsm_x4(ai, sA + 64 * kOzLd + a_off + k0);
#pragma unroll
          for (int e = 0; e < 4; ++e) an[e] = ai[e] ^ 0x80008000u;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint32_t br[4], bi[4];
            ldsm_x4(br, sB + b_off + h * 16 * kOzLd + k0);
            ldsm_x4(bi, sB + 64 * kOzLd + b_off + h * 16 * kOzLd + k0);
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              const int u = 2 * h + v;
              // (ar + i ai)(br + i bi), or (ar - i ai)(br + i bi) when ConjA
              mma_bf16(cr[u], ar, br[2 * v], br[2 * v + 1]);
              mma_bf16(cr[u], ConjA ? ai : an, bi[2 * v], bi[2 * v + 1]);
              mma_bf16(ci[u], ar, bi[2 * v], bi[2 * v + 1]);
              mma_bf16(ci[u], ConjA ? an : ai, br[2 * v], br[2 * v + 1]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            G[u][e][0] += __float2int_rn(cr[u][e]);
            G[u][e][1] += __float2int_rn(ci[u][e]);
          }
        buf ^= 1;
        if (++gcount == 127) {   // keep the int32 sums below 2^31
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              acc[u][e][0] = fma((double)G[u][e][0], scale, acc[u][e][0]);
              acc[u][e][1] = fma((double)G[u][e][1], scale, acc[u][e][1]);
              G[u][e][0] = G[u][e][1] = 0;
            }
          gcount = 0;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        acc[u][e][0] = fma((double)G[u][e][0], scale, acc[u][e][0]);
        acc[u][e][1] = fma((double)G[u][e][1], scale, acc[u][e][1]);
      }
  }
}

__device__ __forceinline__ void oz_tile_accumulate(__nv_bfloat16* sm, const __nv_bfloat16* Asl,
                                                   const __nv_bfloat16* Bsl, int64_t partstride,
                                                   int kp, int i0, int j0, int kt,
                                                   double (&acc)[4][4][2]) {
  oz_tile_acc<kOzSlices, kOzSlices - 1, false>(sm, Asl, Bsl, partstride, kp, i0, j0, kt, acc);
}

// one CTA per 64 x 64 tile of the box's (s+n) x (s+n) Schur update
__global__ void __launch_bounds__(256) k_oz_schur(LevelDev L, int b0, const OzBox* __restrict__ oz,
                                                  const __nv_bfloat16* __restrict__ slices,
                                                  const int* __restrict__ expo) {
  extern __shared__ __align__(16) __nv_bfloat16 sm[];
  __shared__ int rloc[64], rpos[64], cloc[64], cpos[64], rex[64], cex[64];
  const int b = b0 + blockIdx.y;
  const BoxDesc d = L.desc[b];
  const BoxRun run = L.run[b];
  const int s = run.s, r = run.r, n = run.n;
  if (r < kOzMinK) return;   // small inner dimension: fp64 FMA kernel
  const OzBox o = oz[blockIdx.y];
  const int m = s + n;
  const int tms = (m + 63) / 64;
  if ((int)blockIdx.x >= tms * tms) return;
  const int tm = blockIdx.x % tms, tn = blockIdx.x / tms;
  const int i0 = tm * 64, j0 = tn * 64;
  const int kt = (r + 15) & ~15;
  const int* perm = L.iarena + d.idx_off + d.a + d.nmax;
  const int* ndof = L.rows + d.rows_off + 3 * d.qmax;
  const int* npos = ndof + d.nmax;
  const int* nloc = npos + d.nmax;
  const int* ex = expo + o.e_off;
  if (threadIdx.x < 64) {
    int t = threadIdx.x;
    int i = i0 + t, j = j0 + t;
    if (i < s) { rloc[t] = 0; rpos[t] = perm[i]; }
    else if (i < m) { rloc[t] = nloc[i - s]; rpos[t] = npos[i - s]; }
    if (j < s) { cloc[t] = 0; cpos[t] = perm[j]; }
    else if (j < m) { cloc[t] = nloc[j - s]; cpos[t] = npos[j - s]; }
    rex[t] = i < m ? ex[i] : 0;
    cex[t] = j < m ? ex[o.mpad + j] : 0;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int wr = (warp & 3) * 16;
  const int wc = (warp >> 2) * 32;
  double acc[4][4][2];
  oz_tile_accumulate(sm, slices + o.a_off, slices + o.b_off, (int64_t)o.mpad * o.kp, o.kp, i0, j0,
                     kt, acc);
  __syncthreads();
  // epilogue: scale by 2^(E_i + F_j) in fp64 and subtract from Delta
  const int cnt = 1 + d.ncnt;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int li = wr + g + ((e >> 1) ? 8 : 0);
      const int lj = wc + 8 * u + 2 * tq + (e & 1);
      const int i = i0 + li, j = j0 + lj;
      if (i >= m || j >= m) continue;
      const int sc = rex[li] + cex[lj];
      double vr = ldexp(acc[u][e][0], sc);
      double vi = ldexp(acc[u][e][1], sc);
      const int xl = rloc[li], yl = cloc[lj];
      int64_t off = L.pairtab[d.pairtab + (int64_t)xl * cnt + yl];
      if (off < 0) { set_status(L.status, kStatusBound); continue; }
      int ld = xl == 0 ? d.a : L.cur_a0[L.nlist[d.nbeg + xl - 1]];
      double2* pz = L.delta + off + rpos[li] + (int64_t)cpos[lj] * ld;
      double2 cur = *pz;
      *pz = make_double2(cur.x - vr, cur.y - vi);
    }
}

// ---------------------------------------------------------------------------
// Generic exactly-split complex GEMM C <- epi(op(A) op(B)) for the other
// fp64 products of the elimination (same splitting and exact accumulation as
// the Schur update above). A problem supplies the sizes of one box, element
// accessors of op(A) (m x k) and op(B) (k x n), and the epilogue.
// Boxes whose inner dimension is below kOzMinK use the fp64 FMA kernels.

struct ProbW {      // W = X_CR X_RR^{-1}: (s+n) x r x r, stored
  __device__ static bool dims(const BoxDesc& d, const BoxRun& rr, int& m, int& n, int& k) {
    m = rr.s + rr.n; n = rr.r; k = rr.r; return rr.r >= kOzMinK;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, int i, int kk) {
    return L.arena[d.G3_off + i + (int64_t)(rr.s + kk) * (d.a + d.nmax)];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun&, int kk, int j) {
    return L.arena[d.Xinv_off + kk + (int64_t)j * d.a];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun&, int i, int j,
                             double vr, double vi) {
    L.Wbuf[d.W_off + i + (int64_t)j * (d.a + d.nmax)] = make_double2(vr, vi);
  }
};

struct ProbG1 {     // G1[s:a, :] -= T^T G1[0:s, :]: r x (a+n) x s
  __device__ static bool dims(const BoxDesc& d, const BoxRun& rr, int& m, int& n, int& k) {
    m = rr.r; n = d.a + rr.n; k = rr.s; return rr.r > 0 && rr.s >= kOzMinK;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun&, int i, int kk) {
    return L.arena[d.T_off + kk + (int64_t)i * d.a];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun&, int kk, int j) {
    return L.arena[d.G1_off + kk + (int64_t)j * d.a];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, int i, int j,
                             double vr, double vi) {
    double2* c = L.arena + d.G1_off + (rr.s + i) + (int64_t)j * d.a;
    double2 t = *c;
    *c = make_double2(t.x - vr, t.y - vi);
  }
};

struct ProbG3 {     // G3[:, s:a] -= G3[:, 0:s] T: (a+n) x r x s
  __device__ static bool dims(const BoxDesc& d, const BoxRun& rr, int& m, int& n, int& k) {
    m = d.a + rr.n; n = rr.r; k = rr.s; return rr.r > 0 && rr.s >= kOzMinK;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun&, int i, int kk) {
    return L.arena[d.G3_off + i + (int64_t)kk * (d.a + d.nmax)];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun&, int kk, int j) {
    return L.arena[d.T_off + kk + (int64_t)j * d.a];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, int i, int j,
                             double vr, double vi) {
    double2* c = L.arena + d.G3_off + i + (int64_t)(rr.s + j) * (d.a + d.nmax);
    double2 t = *c;
    *c = make_double2(t.x - vr, t.y - vi);
  }
};

// rows of op(A) (y = 0) or columns of op(B) (y = 1) into digit slices
template <class Prob>
__global__ void __launch_bounds__(256) k_ozg_split(LevelDev L, int b0, const OzBox* __restrict__ oz,
                                                   __nv_bfloat16* slices, int* expo) {
  const int b = b0 + blockIdx.z;
  const BoxDesc d = L.desc[b];
  const BoxRun rr = L.run[b];
  int m, n, k;
  if (!Prob::dims(d, rr, m, n, k)) return;
  const OzBox o = oz[blockIdx.z];
  const bool cols = blockIdx.y == 1;
  const int len = cols ? n : m;
  const int lt = (len + 63) & ~63;
  const int kt = (k + 15) & ~15;
  const int i0 = blockIdx.x * 32;
  if (i0 >= lt) return;
  __nv_bfloat16* base = slices + (cols ? o.b_off : o.a_off);
  int* ex = expo + o.e_off + (cols ? o.mpad : 0);
  const int64_t partstride = (int64_t)o.mpad * o.kp;
  const int64_t pstride = 2 * partstride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int rr2 = warp; rr2 < 32; rr2 += 8) {
    const int i = i0 + rr2;
    if (i >= lt) break;
    double mx = 0.0;
    if (i < len)
      for (int kk = lane; kk < k; kk += 32) {
        double2 v = cols ? Prob::B(L, d, rr, kk, i) : Prob::A(L, d, rr, i, kk);
        mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
      }
    for (int o2 = 16; o2 > 0; o2 >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o2));
    const int e = row_exponent(mx);
    if (lane == 0) ex[i] = e;
    for (int kk = lane; kk < kt; kk += 32) {
      double2 v = make_double2(0.0, 0.0);
      if (i < len && kk < k) v = cols ? Prob::B(L, d, rr, kk, i) : Prob::A(L, d, rr, i, kk);
      __nv_bfloat16* dst = base + (int64_t)i * o.kp + kk;
      split_digits(v.x, e, dst, pstride);
      split_digits(v.y, e, dst + partstride, pstride);
    }
  }
}

template <class Prob>
__global__ void __launch_bounds__(256) k_ozg_gemm(LevelDev L, int b0, const OzBox* __restrict__ oz,
                                                  const __nv_bfloat16* __restrict__ slices,
                                                  const int* __restrict__ expo) {
  extern __shared__ __align__(16) __nv_bfloat16 sm[];
  __shared__ int rex[64], cex[64];
  const int b = b0 + blockIdx.y;
  const BoxDesc d = L.desc[b];
  const BoxRun rr = L.run[b];
  int m, n, k;
  if (!Prob::dims(d, rr, m, n, k)) return;
  const OzBox o = oz[blockIdx.y];
  const int tms = (m + 63) / 64, tns = (n + 63) / 64;
  if ((int)blockIdx.x >= tms * tns) return;
  const int i0 = (blockIdx.x % tms) * 64, j0 = (blockIdx.x / tms) * 64;
  const int kt = (k + 15) & ~15;
  const int* ex = expo + o.e_off;
  if (threadIdx.x < 64) {
    int t = threadIdx.x;
    rex[t] = i0 + t < m ? ex[i0 + t] : 0;
    cex[t] = j0 + t < n ? ex[o.mpad + j0 + t] : 0;
  }
  double acc[4][4][2];
  oz_tile_accumulate(sm, slices + o.a_off, slices + o.b_off, (int64_t)o.mpad * o.kp, o.kp, i0, j0,
                     kt, acc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int wr = (warp & 3) * 16, wc = (warp >> 2) * 32;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int li = wr + g + ((e >> 1) ? 8 : 0);
      const int lj = wc + 8 * u + 2 * tq + (e & 1);
      const int i = i0 + li, j = j0 + lj;
      if (i >= m || j >= n) continue;
      const int sc = rex[li] + cex[lj];
      Prob::epi(L, d, rr, i, j, ldexp(acc[u][e][0], sc), ldexp(acc[u][e][1], sc));
    }
}

template <class Prob>
static void launch_ozg(const char* name, const LevelDev& L, int b0, int nb, const OzBox* oz,
                       __nv_bfloat16* sl, int* expo, int mmax, int nmax, cudaStream_t st) {
  const size_t smem = (size_t)4 * kOzStage * sizeof(__nv_bfloat16);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_ozg_gemm<Prob>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  int big = std::max(mmax, nmax);
  dim3 gs((unsigned)((big + 63) / 64 * 2), 2, nb);
  FMMLU_LAUNCH("oz_split", st, k_ozg_split<Prob><<<gs, 256, 0, st>>>(L, b0, oz, sl, expo));
  dim3 gm((unsigned)(((mmax + 63) / 64) * ((nmax + 63) / 64)), nb);
  FMMLU_LAUNCH(name, st, k_ozg_gemm<Prob><<<gm, 256, smem, st>>>(L, b0, oz, sl, expo));
}

void launch_oz_elim_gemms(const LevelDev& L, int b0, int nb, const OzBoxHost* d_oz, void* slices,
                          int* expo, int amax, int nmax_max, int which, cudaStream_t st) {
  if (nb <= 0) return;
  __nv_bfloat16* sl = reinterpret_cast<__nv_bfloat16*>(slices);
  if (which == 0) launch_ozg<ProbG1>("gemm_g1_tc", L, b0, nb, d_oz, sl, expo, amax, amax + nmax_max, st);
  if (which == 1) launch_ozg<ProbG3>("gemm_g3_tc", L, b0, nb, d_oz, sl, expo, amax + nmax_max, amax, st);
  if (which == 2) launch_ozg<ProbW>("gemm_w_tc", L, b0, nb, d_oz, sl, expo, amax + nmax_max, amax, st);
}

size_t oz_slice_elems(int a, int nmax) {
  int64_t mpad = ((int64_t)a + nmax + 63) & ~63;
  int64_t kp = ((int64_t)a + 15) & ~15;
  return (size_t)(2 * kOzSlices * 2 * mpad * kp);   // W and X_RC, both parts
}

void plan_oz_box(int a, int nmax, int64_t& slice_off, int64_t& expo_off, OzBoxHost& out) {
  int64_t mpad = ((int64_t)a + nmax + 63) & ~63;
  int64_t kp = ((int64_t)a + 15) & ~15;
  out.a_off = slice_off;
  out.b_off = slice_off + (int64_t)kOzSlices * 2 * mpad * kp;
  out.e_off = expo_off;
  out.mpad = (int)mpad;
  out.kp = (int)kp;
  slice_off += 2 * (int64_t)kOzSlices * 2 * mpad * kp;
  expo_off += 2 * mpad;
}

void launch_oz_schur(const LevelDev& L, int b0, int nb, const OzBoxHost* d_oz, void* slices,
                     int* expo, int amax, int nmax_max, cudaStream_t st) {
  if (nb <= 0) return;
  const OzBox* oz = d_oz;
  __nv_bfloat16* sl = reinterpret_cast<__nv_bfloat16*>(slices);
  int mmax = amax + nmax_max;
  dim3 gs((unsigned)((mmax + 63) / 64 * 2), 2, nb);
  FMMLU_LAUNCH("oz_split", st, k_oz_split<<<gs, 256, 0, st>>>(L, b0, oz, sl, expo));
  int t = (mmax + 63) / 64;
  dim3 gm((unsigned)(t * t), nb);
  const size_t smem = (size_t)4 * kOzStage * sizeof(__nv_bfloat16);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_oz_schur, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  FMMLU_LAUNCH("schur_tc", st, k_oz_schur<<<gm, 256, smem, st>>>(L, b0, oz, sl, expo));
}

// ---------------------------------------------------------------------------
// Gram matrix G = M^H M of a box's ID matrix (m x a, column-major, ld mmax).
// Each column of M is one row of digit slices (the contraction runs over the
// rows of M, contiguous in memory), scaled by a power of two from its largest
// component. complex128 columns take 7 digits and the pairs p + q <= 6 (the
// omitted pairs are below 2^-56 of the column maxima); complex64 columns take
// 4 digits and the pairs p + q <= 4 (below 2^-40). Every digit product and
// every 128-term block sum is exact; the only roundings are fp64 additions.

template <int NS, typename C>
__global__ void __launch_bounds__(256) k_gram_split(LevelDev L, int b0,
                                                    const GramBoxHost* __restrict__ gb,
                                                    __nv_bfloat16* slices, int* expo) {
  const int b = b0 + blockIdx.y;
  const BoxDesc d = L.desc[b];
  const GramBoxHost g = gb[b];
  const int a = d.a;
  const int m = 2 * L.run[b].nq + 2 * L.n_proxy;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * 8 + warp;       // column of M, row of the slices
  if (k >= g.apad) return;
  const int kt = (m + 15) & ~15;
  const C* col = reinterpret_cast<const C*>(L.Mbuf) + d.M_off + (int64_t)k * d.mmax;
  double mx = 0.0;
  if (k < a)
    for (int i = lane; i < m; i += 32) {
      double2 v = to_d2(col[i]);
      mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
    }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const bool bad = !(mx <= 1.7976931348623157e308);   // inf or NaN in the column
  if (bad) {
    if (lane == 0) set_status(L.status, kStatusNonfinite);
    mx = 0.0;
  }
  const int e = row_exponent(mx);
  if (lane == 0) expo[g.e_off + k] = e;
  const int64_t partstride = (int64_t)g.apad * g.kp;
  const int64_t pstride = 2 * partstride;
  __nv_bfloat16* dst = slices + g.sl_off + (int64_t)k * g.kp;
  for (int i = lane; i < kt; i += 32) {
    double2 v = make_double2(0.0, 0.0);
    if (k < a && i < m && !bad) v = to_d2(col[i]);
    split_digits_n<NS>(v.x, e, dst + i, pstride);
    split_digits_n<NS>(v.y, e, dst + partstride + i, pstride);
  }
}

// one CTA per 64 x 64 tile (tm <= tn) of the upper triangle; the lower one is
// written as the conjugate transpose
template <int NS, int DMAX>
__global__ void __launch_bounds__(256) k_gram(LevelDev L, int b0, const GramBoxHost* __restrict__ gb,
                                              const __nv_bfloat16* __restrict__ slices,
                                              const int* __restrict__ expo, double2* gbuf) {
  extern __shared__ __align__(16) __nv_bfloat16 sm[];
  __shared__ int rex[64], cex[64];
  const int b = b0 + blockIdx.y;
  const BoxDesc d = L.desc[b];
  const GramBoxHost g = gb[b];
  const int a = d.a;
  const int m = 2 * L.run[b].nq + 2 * L.n_proxy;
  const int ta = (a + 63) / 64;
  const int x = blockIdx.x;
  if (x >= ta * (ta + 1) / 2) return;
  int tn = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
  while ((tn + 1) * (tn + 2) / 2 <= x) ++tn;
  while (tn * (tn + 1) / 2 > x) --tn;
  const int tm = x - tn * (tn + 1) / 2;
  const int i0 = tm * 64, j0 = tn * 64;
  const int kt = (m + 15) & ~15;
  if (threadIdx.x < 64) {
    rex[threadIdx.x] = expo[g.e_off + i0 + threadIdx.x];
    cex[threadIdx.x] = expo[g.e_off + j0 + threadIdx.x];
  }
  const __nv_bfloat16* sl = slices + g.sl_off;
  double acc[4][4][2];
  oz_tile_acc<NS, DMAX, true>(sm, sl, sl, (int64_t)g.apad * g.kp, g.kp, i0, j0, kt, acc);
  double2* G = gbuf + g.G_off;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, tq = lane & 3;
  const int wr = (warp & 3) * 16, wc = (warp >> 2) * 32;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int li = wr + gq + ((e >> 1) ? 8 : 0);
      const int lj = wc + 8 * u + 2 * tq + (e & 1);
      const int i = i0 + li, j = j0 + lj;
      if (i >= a || j >= a) continue;
      const int sc = rex[li] + cex[lj];
      const double vr = ldexp(acc[u][e][0], sc);
      const double vi = i == j ? 0.0 : ldexp(acc[u][e][1], sc);
      G[i + (int64_t)j * a] = make_double2(vr, vi);
      if (tm != tn) G[j + (int64_t)i * a] = make_double2(vr, -vi);
    }
}

constexpr int kGramNS64 = 7, kGramNS32 = 4;

void plan_gram_box(int a, int mmax, bool fp32, int64_t& slice_off, int64_t& expo_off,
                   int64_t& g_off, GramBoxHost& out) {
  const int ns = fp32 ? kGramNS32 : kGramNS64;
  out.apad = (a + 63) & ~63;
  out.kp = (mmax + 15) & ~15;
  out.sl_off = slice_off;
  out.e_off = expo_off;
  out.G_off = g_off;
  slice_off += (int64_t)ns * 2 * out.apad * out.kp;
  expo_off += out.apad;
  g_off += 2 * (int64_t)a * a;
}

void launch_gram(const LevelDev& L, int b0, int nb, const GramBoxHost* d_gb, void* slices,
                 int* expo, double2* gbuf, int amax, int mmax, bool fp32, cudaStream_t st) {
  if (nb <= 0) return;
  __nv_bfloat16* sl = reinterpret_cast<__nv_bfloat16*>(slices);
  const int apad = (amax + 63) & ~63;
  dim3 gs((unsigned)(apad / 8), nb);
  const size_t smem = (size_t)4 * kOzStage * sizeof(__nv_bfloat16);
  const int ta = apad / 64;
  dim3 gm((unsigned)(ta * (ta + 1) / 2), nb);
  (void)mmax;
  if (fp32) {
    FMMLU_LAUNCH("gram_split", st,
                 (k_gram_split<kGramNS32, float2><<<gs, 256, 0, st>>>(L, b0, d_gb, sl, expo)));
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_gram<kGramNS32, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      attr = true;
    }
    FMMLU_LAUNCH("gram", st,
                 (k_gram<kGramNS32, 4><<<gm, 256, smem, st>>>(L, b0, d_gb, sl, expo, gbuf)));
  } else {
    FMMLU_LAUNCH("gram_split", st,
                 (k_gram_split<kGramNS64, double2><<<gs, 256, 0, st>>>(L, b0, d_gb, sl, expo)));
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_gram<kGramNS64, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      attr = true;
    }
    FMMLU_LAUNCH("gram", st,
                 (k_gram<kGramNS64, 6><<<gm, 256, smem, st>>>(L, b0, d_gb, sl, expo, gbuf)));
  }
}

}  // namespace fmmlu
