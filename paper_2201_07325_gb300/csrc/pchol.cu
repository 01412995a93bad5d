// Greedy pivoted Cholesky of the Gram matrix G = M^H M of a box's ID matrix.
//
// The ID of Def. ID picks columns of M greedily: step j takes the remaining
// column whose component orthogonal to the columns already taken is largest,
// and the selection stops once that norm is at most eps times the first one.
// Those squared norms are the diagonal of the Schur complement of G, so the
// same selection runs on G alone: step j takes the column p of largest
// residual d_p, sets R_jj = sqrt(d_p) and
//     R_jk = (G_pk - sum_{i<j} conj(R_ip) R_ik) / R_jj      (k not yet taken)
// and lowers d_k by |R_jk|^2. In exact arithmetic R is the R factor of CPQR of
// M up to unimodular row scalings, which cancel in T = R_11^{-1} R_12.
//
// Distribution: P CTAs per box, column k owned by CTA k mod P, R stored by
// columns next to G. Each step ends with one bounded per-box barrier: every
// CTA publishes the largest residual among its columns and all CTAs take the
// same pivot from the P candidates (ties to the lowest index). With P > 1 the
// launch is cooperative (all CTAs co-resident); with P = 1 every barrier is
// passed at once. Every wait is bounded (coop.cuh).
#include "coop.cuh"

namespace fmmlu {

constexpr int kPcThreads = 256;
constexpr int kPcWarps = kPcThreads / 32;

struct PcCand {
  double val;
  int idx;
  int pad_;
};

__device__ __forceinline__ bool pc_better(double v, int i, double bv, int bi) {
  return v > bv || (v == bv && i < bi);
}

__device__ __forceinline__ void pc_warp_best(double& bv, int& bi) {
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (pc_better(ov, oi, bv, bi)) { bv = ov; bi = oi; }
  }
}

// sum over the 8 lanes of a segment (lanes 8c .. 8c+7)
__device__ __forceinline__ double pc_seg8_sum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

size_t pchol_smem(int amax) {
  // colp (double2), piv, pos (int), residuals (double), per-warp solve columns
  return (size_t)amax * (16 + 4 + 4 + 8) + (size_t)kPcWarps * amax * 16;
}

// The CTAs of a box are parts[] entries: P = 1, one CTA per box with its
// candidates and barriers in shared memory; P > 1, a cooperative launch with
// candidates and bounded barriers in global memory.
__global__ void __launch_bounds__(kPcThreads) k_pchol(LevelDev L, const CpqrPart* __restrict__ parts,
                                                      unsigned char* scratch,
                                                      const GramBoxHost* __restrict__ gb,
                                                      double2* gbuf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const CpqrPart me = parts[blockIdx.x];
  const int b = me.box;
  const int rank = me.rank;
  const int P = me.P;
  const BoxDesc d = L.desc[b];
  const int a = d.a;
  const int m = 2 * L.run[b].nq + 2 * L.n_proxy;
  const GramBoxHost gx = gb[b];
  const double2* G = gbuf + gx.G_off;                  // a x a, Hermitian, column-major
  double2* Rc = gbuf + gx.G_off + (int64_t)a * a;      // column k holds R_0k, R_1k, ...
  unsigned char* sc = scratch + me.scratch_off;
  unsigned* ctr = reinterpret_cast<unsigned*>(sc);
  int* abort_flag = reinterpret_cast<int*>(sc + 4);
  // candidates [2][P] by step parity: in global memory when several CTAs
  // share the box, in shared memory when the CTA is alone
  __shared__ PcCand s_cand[2];
  PcCand* cand = P == 1 ? s_cand : reinterpret_cast<PcCand*>(sc + 16);
  double2* colp = reinterpret_cast<double2*>(smem_raw);
  int* piv = reinterpret_cast<int*>(colp + a);
  int* pos = piv + a;
  double* dres = reinterpret_cast<double*>(pos + a);  // owned columns; -1 once taken
  double2* xs = reinterpret_cast<double2*>(dres + a);  // kPcWarps columns of length a
  __shared__ int s_piv, s_stop;
  __shared__ double s_nrm, s_r11;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nown = a > rank ? (a - rank + P - 1) / P : 0;
  const double eps = L.eps;
  unsigned nbar = 0;
#define BARRIER()                                                                   \
  do {                                                                              \
    ++nbar;                                                                         \
    if (P == 1) {                                                                   \
      __syncthreads();                                                              \
    } else if (!box_barrier(ctr, nbar * (unsigned)P, abort_flag, L.status)) {       \
      return;                                                                       \
    }                                                                               \
  } while (0)

  auto publish = [&](int par) {
    if (warp != 0) return;
    double bv = -1.0;
    int bi = a;
    for (int t = lane; t < nown; t += 32) {
      double v = dres[t];
      if (v < 0.0) continue;                 // taken
      if (!(v == v)) v = INFINITY;           // NaN: picked, then reported
      const int k = rank + P * t;
      if (pc_better(v, k, bv, bi)) { bv = v; bi = k; }
    }
    pc_warp_best(bv, bi);
    if (lane == 0) {
      if (P == 1) {
        cand[par].val = bv;
        cand[par].idx = bi;
      } else {
        stcg(&cand[par * P + rank].val, bv);
        stcg(&cand[par * P + rank].idx, bi);
      }
    }
  };

  for (int t = tid; t < nown; t += blockDim.x) {
    const int k = rank + P * t;
    dres[t] = G[k + (int64_t)k * a].x;
  }
  __syncthreads();
  publish(0);
  BARRIER();
  const int steps = min(m, a);
  int s = steps;
  const int grp = tid >> 3, sl = tid & 7, ngrp = blockDim.x >> 3;
  for (int j = 0; j < steps; ++j) {
    const int par = j & 1;
    if (warp == 0) {
      double bv = -1.0;
      int bi = a;
      for (int c = lane; c < P; c += 32) {
        double v;
        int i;
        if (P == 1) {
          v = cand[par].val;
          i = cand[par].idx;
        } else {
          v = ldcg(&cand[par * P + c].val);
          i = ldcg(&cand[par * P + c].idx);
        }
        if (pc_better(v, i, bv, bi)) { bv = v; bi = i; }
      }
      pc_warp_best(bv, bi);
      if (lane == 0) {
        const double nrm = sqrt(bv);
        if (j == 0) s_r11 = nrm;
        int stop = bi >= a ? 1 : 0;
        if (!(nrm < INFINITY)) {
          if (rank == 0) set_status(L.status, kStatusNonfinite);
          stop = 1;
        }
        if (!(nrm > eps * s_r11) || nrm == 0.0) stop = 1;
        s_stop = stop;
        s_piv = bi;
        s_nrm = nrm;
      }
    }
    __syncthreads();
    if (s_stop) { s = j; break; }
    const int p = s_piv;
    const double nrm = s_nrm, inv = 1.0 / nrm;
    if (tid == 0) piv[j] = p;
    for (int i = tid; i < j; i += blockDim.x) colp[i] = ldcg(Rc + (int64_t)p * a + i);
    __syncthreads();
    // row j of R over the owned columns, one 8-lane segment per column
    for (int t0 = 0; t0 < nown; t0 += ngrp) {
      const int t = t0 + grp;
      const int k = rank + P * t;
      const bool act = t < nown && !(dres[t] < 0.0);
      double2 acc = make_double2(0.0, 0.0);
      if (act && k != p) {
        const double2* rk = Rc + (int64_t)k * a;
        for (int i = sl; i < j; i += 8) cfma_cj(acc, colp[i], ldcg(rk + i));
      }
      acc.x = pc_seg8_sum(acc.x);
      acc.y = pc_seg8_sum(acc.y);
      if (act && sl == 0) {
        if (k == p) {
          stcg(Rc + (int64_t)p * a + j, make_double2(nrm, 0.0));
          dres[t] = -1.0;
        } else {
          const double2 gkp = G[k + (int64_t)p * a];          // G_pk = conj(G_kp)
          const double2 rjk = make_double2((gkp.x - acc.x) * inv, (-gkp.y - acc.y) * inv);
          stcg(Rc + (int64_t)k * a + j, rjk);
          const double v = dres[t] - cabs2(rjk);
          dres[t] = v < 0.0 ? 0.0 : v;
        }
      }
    }
    __syncthreads();
    publish(par ^ 1);
    BARRIER();
  }
#undef BARRIER
  // taken columns in pivot order, the others by increasing index
  __syncthreads();
  for (int k = tid; k < a; k += blockDim.x) pos[k] = -1;
  __syncthreads();
  for (int i = tid; i < s; i += blockDim.x) pos[piv[i]] = i;
  __syncthreads();
  int* red = reinterpret_cast<int*>(colp);
  if (tid == 0) {
    int c = 0;
    for (int k = 0; k < a; ++k)
      if (pos[k] < 0) red[c++] = k;
  }
  __syncthreads();
  const int r = a - s;
  // T = R_11^{-1} R_12 by back substitution, one warp per column of T
  double2* T = L.arena + d.T_off;
  double2* x = xs + (int64_t)warp * a;
  for (int c = rank + P * warp; c < r; c += P * kPcWarps) {
    const double2* src = Rc + (int64_t)red[c] * a;
    for (int i = lane; i < s; i += 32) x[i] = ldcg(src + i);
    __syncwarp();
    for (int l = s - 1; l >= 0; --l) {
      const double2* cl = Rc + (int64_t)piv[l] * a;      // column l of R_11 (rows 0 .. l)
      const double dl = ldcg(cl + l).x;
      const double2 xl = x[l];
      const double2 tl = make_double2(xl.x / dl, xl.y / dl);
      __syncwarp();
      if (lane == 0) x[l] = tl;
      for (int i = lane; i < l; i += 32) {
        double2 v = x[i];
        cfms(v, ldcg(cl + i), tl);
        x[i] = v;
      }
      __syncwarp();
    }
    for (int i = lane; i < s; i += 32) T[i + (int64_t)c * a] = x[i];
    __syncwarp();
  }
  if (rank != 0) return;
  int* idx = L.iarena + d.idx_off;
  int* pv = idx + a + d.nmax;
  const int base = L.cur_off[d.cur];
  const int* ndof = L.rows + d.rows_off + 3 * d.qmax;
  const int n = L.run[b].n;
  for (int k = tid; k < a; k += blockDim.x) {
    const int p = k < s ? piv[k] : red[k - s];
    pv[k] = p;
    const int dof = L.act_dof[base + p];
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

size_t pchol_scratch_bytes(int P) {
  size_t bytes = 16 + 2 * (size_t)P * sizeof(PcCand);
  return (bytes + 255) & ~(size_t)255;
}

int pchol_capacity(int amax) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t sm = pchol_smem(amax);
  cudaFuncSetAttribute(k_pchol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pchol, kPcThreads, sm);
  return occ * sms;
}

cudaError_t launch_pchol(const LevelDev& L, const CpqrPart* d_parts, int nparts,
                         unsigned char* scratch, const GramBoxHost* d_gb, double2* gbuf, int amax,
                         bool cooperative, cudaStream_t st) {
  if (nparts <= 0) return cudaSuccess;
  const size_t sm = pchol_smem(amax);
  cudaError_t e =
      cudaFuncSetAttribute(k_pchol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  if (!cooperative) {
    FMMLU_LAUNCH("pchol", st,
                 (k_pchol<<<nparts, kPcThreads, sm, st>>>(L, d_parts, scratch, d_gb, gbuf)));
    return cudaGetLastError();
  }
  LevelDev Lc = L;
  const CpqrPart* pp = d_parts;
  unsigned char* sp = scratch;
  const GramBoxHost* gp = d_gb;
  double2* gq = gbuf;
  void* args[] = {&Lc, &pp, &sp, &gp, &gq};
  FMMLU_LAUNCH("pchol", st,
               e = cudaLaunchCooperativeKernel((const void*)k_pchol, dim3(nparts),
                                               dim3(kPcThreads), args, sm, st));
  return e;
}

}  // namespace fmmlu
