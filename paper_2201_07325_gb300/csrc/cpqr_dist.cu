// Greedy column-pivoted QR of the ID matrix, distributed over the rows.
//
// The same algorithm as k_cpqr (Def. ID, greedy CPQR: pivot = remaining column
// of largest norm, ties to the lowest index, stop when |R_jj| <= eps |R_11|,
// T = R_11^{-1} R_12), but one box is processed by P cooperating CTAs: CTA c
// owns the contiguous rows [c*chunk, (c+1)*chunk) of the box's m x a matrix.
// Per step j:
//   1. every CTA reads the reduced column norms, picks the same pivot, swaps
//      columns j and p in its rows, forms partial dots of the pivot column
//      below row j with the trailing columns; the owner of row j publishes it;
//   2. CTA c reduces the partial dots of the columns k = c (mod P);
//   3. every CTA forms the reflector from the published row and the reduced
//      norm, updates its rows and forms partial norms of rows > j;
//   4. CTA c reduces the partial norms of its columns.
// With P <= kRedundantP every CTA instead reduces all partial dots and norms
// itself (steps 2 and 4 vanish): two barriers per step instead of four.
// Steps are separated by per-box barriers (a counter in global memory). All
// CTAs of a launch are co-resident (cooperative launch). Every wait is
// bounded: after kSpinLimit polls the box's abort flag is raised, the status
// word gets kStatusTimeout and all CTAs of the box return.
#include <algorithm>
#include <vector>

#include "coop.cuh"

namespace fmmlu {

constexpr int kDistThreads = 256;
constexpr int kRedundantP = 32;
// sum over the 8 lanes of a segment (lanes 8c .. 8c+7)
template <typename T> __device__ __forceinline__ T seg8_sum(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

template <typename Rl>
__global__ void __launch_bounds__(kDistThreads) k_cpqr_dist(LevelDev L,
                                                            const CpqrPart* __restrict__ parts,
                                                            unsigned char* scratch) {
  using C = typename CT<Rl>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const CpqrPart me = parts[blockIdx.x];
  const int b = me.box, rank = me.rank, P = me.P;
  const BoxDesc d = L.desc[b];
  const int a = d.a;
  const int nq = L.run[b].nq;
  const int m = 2 * nq + 2 * L.n_proxy;
  const int64_t ld = d.mmax;
  C* M = reinterpret_cast<C*>(L.Mbuf) + d.M_off;
  unsigned char* sc = scratch + me.scratch_off;
  unsigned* ctr = reinterpret_cast<unsigned*>(sc);
  int* abort_flag = reinterpret_cast<int*>(sc + 4);
  C* part_dot = reinterpret_cast<C*>(sc + 16);
  C* dot_full = part_dot + (int64_t)P * a;
  C* rowj = dot_full + a;
  Rl* part_norm = reinterpret_cast<Rl*>(rowj + a);
  Rl* norm_full = part_norm + (int64_t)P * a;
  C* w = reinterpret_cast<C*>(smem_raw);
  Rl* norms = reinterpret_cast<Rl*>(w + a);
  int* perm = reinterpret_cast<int*>(norms + a);
  __shared__ int s_piv, s_rank;
  __shared__ Rl s_r11, s_tau;
  __shared__ C s_v0, s_alpha;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const Rl eps = (Rl)L.eps;
  const int chunk = ((m + P - 1) / P + 31) & ~31;   // whole warps of rows
  const int r0 = min(m, rank * chunk), r1 = min(m, r0 + chunk);
  unsigned nbar = 0;
#define BARRIER()                                                                   \
  do {                                                                              \
    ++nbar;                                                                         \
    if (!box_barrier(ctr, nbar * (unsigned)P, abort_flag, L.status)) return;       \
  } while (0)

  // column work: each warp takes 4 columns at a time, 8 lanes per column
  const int sub = lane >> 3, sl = lane & 7;
  for (int k = tid; k < a; k += blockDim.x) perm[k] = k;
  for (int kk = 4 * warp; kk < a; kk += 4 * nw) {
    const int k = kk + sub;
    Rl acc = 0;
    if (k < a)
      for (int i = r0 + sl; i < r1; i += 8) cnorm_acc(acc, M[i + k * ld]);
    acc = seg8_sum(acc);
    if (sl == 0 && k < a) stcg(part_norm + (int64_t)rank * a + k, acc);
  }
  BARRIER();
  const bool redundant = P <= kRedundantP;
  if (!redundant) {
    for (int k = rank + P * tid; k < a; k += P * blockDim.x) {
      Rl s = 0;
      for (int c = 0; c < P; ++c) s += ldcg(part_norm + (int64_t)c * a + k);
      stcg(norm_full + k, s);
    }
    BARRIER();
  }
  if (tid == 0) s_rank = min(m, a);
  const int steps = min(m, a);
  for (int j = 0; j < steps; ++j) {
    if (redundant) {
      for (int k = j + tid; k < a; k += blockDim.x) {
        Rl s = 0;
        for (int c = 0; c < P; ++c) s += ldcg(part_norm + (int64_t)c * a + k);
        norms[k] = s;
      }
    } else {
      for (int k = j + tid; k < a; k += blockDim.x) norms[k] = ldcg(norm_full + k);
    }
    __syncthreads();
    if (warp == 0) {
      Rl best = (Rl)-1;
      int bi = a;
      for (int k = j + lane; k < a; k += 32) {
        Rl v = norms[k];
        if (!(v == v)) v = (Rl)INFINITY;
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
        if (!(nrm < (Rl)INFINITY) && rank == 0) set_status(L.status, kStatusNonfinite);
        if (!(nrm > eps * s_r11) || nrm == (Rl)0 || !(nrm < (Rl)INFINITY)) s_rank = j;
      }
    }
    __syncthreads();
    if (s_rank == j) break;
    const int p = s_piv;
    if (p != j) {
      for (int i = r0 + tid; i < r1; i += blockDim.x) {
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
    const int lo = max(r0, j + 1);
    for (int kk = j + 1 + 4 * warp; kk < a; kk += 4 * nw) {
      const int k = kk + sub;
      C acc = mk((Rl)0, (Rl)0);
      if (k < a)
        for (int i = lo + sl; i < r1; i += 8) cfma_cj(acc, M[i + j * ld], M[i + k * ld]);
      acc.x = seg8_sum(acc.x);
      acc.y = seg8_sum(acc.y);
      if (sl == 0 && k < a) stcg(part_dot + (int64_t)rank * a + k, acc);
    }
    const bool owner = r0 <= j && j < r1;
    if (owner)
      for (int k = j + tid; k < a; k += blockDim.x) stcg(rowj + k, M[j + k * ld]);
    BARRIER();
    if (!redundant) {
      for (int k0 = j + 1; k0 < a; k0 += P * blockDim.x) {
        // columns k = j+1 .. a-1 with (k - j - 1) % P == rank
        int k = k0 + rank + P * tid;
        if (k < a) {
          C s = mk((Rl)0, (Rl)0);
          for (int c = 0; c < P; ++c) s = cadd(s, ldcg(part_dot + (int64_t)c * a + k));
          stcg(dot_full + k, s);
        }
      }
      BARRIER();
    }
    if (tid == 0) {
      C x0 = ldcg(rowj + j);
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
    for (int k = j + 1 + tid; k < a; k += blockDim.x) {
      C wk;
      if (redundant) {
        wk = mk((Rl)0, (Rl)0);
        for (int c = 0; c < P; ++c) wk = cadd(wk, ldcg(part_dot + (int64_t)c * a + k));
      } else {
        wk = ldcg(dot_full + k);
      }
      cfma_cj(wk, v0, ldcg(rowj + k));
      w[k] = mk(tau * wk.x, tau * wk.y);
    }
    __syncthreads();
    for (int kk = j + 1 + 4 * warp; kk < a; kk += 4 * nw) {
      const int k = kk + sub;
      Rl acc = 0;
      if (k < a) {
        const C tw = w[k];
        for (int i = lo + sl; i < r1; i += 8) {
          C t = M[i + k * ld];
          cfms(t, M[i + j * ld], tw);
          M[i + k * ld] = t;
          cnorm_acc(acc, t);
        }
      }
      acc = seg8_sum(acc);
      if (sl == 0 && k < a) stcg(part_norm + (int64_t)rank * a + k, acc);
    }
    if (owner) {
      for (int k = j + 1 + tid; k < a; k += blockDim.x) M[j + k * ld] = csub(M[j + k * ld], cmul(v0, w[k]));
      if (tid == 0) M[j + j * ld] = s_alpha;
    }
    BARRIER();
    if (!redundant) {
      for (int k0 = j + 1; k0 < a; k0 += P * blockDim.x) {
        int k = k0 + rank + P * tid;
        if (k < a) {
          Rl s = 0;
          for (int c = 0; c < P; ++c) s += ldcg(part_norm + (int64_t)c * a + k);
          stcg(norm_full + k, s);
        }
      }
      BARRIER();
    }
  }
#undef BARRIER
  __syncthreads();
  const int s = s_rank;
  const int r = a - s;
  // T = R11^{-1} R12: column c = rank + P * i handled by one warp of CTA rank
  double2* T = L.arena + d.T_off;
  for (int c = rank + P * warp; c < r; c += P * nw) {
    C* col = M + (int64_t)(s + c) * ld;
    for (int i = s - 1; i >= 0; --i) {
      __syncwarp();
      C ti = cdiv(ldcg(col + i), ldcg(M + i + (int64_t)i * ld));
      __syncwarp();
      if (lane == 0) stcg(col + i, ti);
      for (int l = lane; l < i; l += 32) stcg(col + l, csub(ldcg(col + l), cmul(ldcg(M + l + (int64_t)i * ld), ti)));
    }
    __syncwarp();
    for (int i = lane; i < s; i += 32) T[i + (int64_t)c * a] = to_d2(ldcg(col + i));
  }
  if (rank != 0) return;
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

static size_t dist_smem(int amax, bool fp32) {
  size_t c = fp32 ? 8 : 16, rl = fp32 ? 4 : 8;
  return (size_t)amax * (c + rl + 4) + 16;
}

size_t cpqr_dist_scratch_bytes(int P, int a, bool fp32) {
  size_t c = fp32 ? 8 : 16, rl = fp32 ? 4 : 8;
  size_t bytes = 16 + c * ((size_t)P * a + 2 * (size_t)a) + rl * ((size_t)P * a + a);
  return (bytes + 255) & ~(size_t)255;
}

int cpqr_dist_capacity(int amax, bool fp32) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  size_t sm = dist_smem(amax, fp32);
  if (fp32) {
    cudaFuncSetAttribute(k_cpqr_dist<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cpqr_dist<float>, kDistThreads, sm);
  } else {
    cudaFuncSetAttribute(k_cpqr_dist<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cpqr_dist<double>, kDistThreads, sm);
  }
  return occ * sms;
}

cudaError_t launch_cpqr_dist(const LevelDev& L, const CpqrPart* d_parts, int nparts,
                             unsigned char* scratch, int amax, bool fp32, cudaStream_t st) {
  size_t sm = dist_smem(amax, fp32);
  // the attribute is per function: set it for this launch's size
  cudaError_t ea = fp32 ? cudaFuncSetAttribute(k_cpqr_dist<float>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                        : cudaFuncSetAttribute(k_cpqr_dist<double>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (ea != cudaSuccess) return ea;
  LevelDev Lc = L;
  const CpqrPart* pp = d_parts;
  unsigned char* sp = scratch;
  void* args[] = {&Lc, &pp, &sp};
  cudaError_t e = cudaSuccess;
  FMMLU_LAUNCH("cpqr", st,
               e = cudaLaunchCooperativeKernel(
                   fp32 ? (const void*)k_cpqr_dist<float> : (const void*)k_cpqr_dist<double>,
                   dim3(nparts), dim3(kDistThreads), args, sm, st));
  return e;
}

}  // namespace fmmlu
