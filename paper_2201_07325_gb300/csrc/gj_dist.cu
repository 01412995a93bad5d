// X_RR^{-1} by Gauss-Jordan elimination with partial pivoting, with the
// columns of one box's r x r matrix spread cyclically over P cooperating CTAs
// (column c belongs to CTA c mod P). Per step j the owner of column j picks
// the pivot row p (largest modulus at or below j, ties to the lowest index)
// and publishes the column with rows j and p exchanged (double-buffered by the
// parity of j); after one barrier every CTA exchanges rows j and p in its own
// columns, scales row j by the pivot's inverse and eliminates column j from
// the other rows. The in-place result is the inverse with its columns
// permuted by the row interchanges; each CTA writes its columns to their final
// positions through a scratch copy. Same arithmetic as the one-CTA
// gauss_jordan in linalg.cu. Launch: cooperative; waits bounded (coop.cuh).
#include "coop.cuh"

namespace fmmlu {

constexpr int kGjThreads = 256;

__global__ void __launch_bounds__(kGjThreads) k_gj_dist(LevelDev L,
                                                        const CpqrPart* __restrict__ parts,
                                                        unsigned char* scratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const CpqrPart me = parts[blockIdx.x];
  const int b = me.box, rank = me.rank, P = me.P;
  const BoxDesc d = L.desc[b];
  const int r = L.run[b].r;
  if (r == 0) return;
  const int64_t ld = d.a;
  double2* X = L.arena + d.Xinv_off;
  unsigned char* sc = scratch + me.scratch_off;
  unsigned* ctr = reinterpret_cast<unsigned*>(sc);
  int* abort_flag = reinterpret_cast<int*>(sc + 4);
  int* pivbuf = reinterpret_cast<int*>(sc + 8);          // 2 ints
  double2* colbuf = reinterpret_cast<double2*>(sc + 16); // 2 x a
  double2* Y = colbuf + 2 * (int64_t)d.a;                 // a x a (ld a)
  double2* tc = reinterpret_cast<double2*>(smem_raw);     // a
  int* ipiv = reinterpret_cast<int*>(tc + d.a);           // a
  int* idx = ipiv + d.a;                                  // a
  __shared__ double s_best[32];
  __shared__ int s_bi[32];
  __shared__ double2 s_inv;
  __shared__ int s_p;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  unsigned nbar = 0;
#define BARRIER()                                                                   \
  do {                                                                              \
    ++nbar;                                                                         \
    if (!box_barrier(ctr, nbar * (unsigned)P, abort_flag, L.status)) return;       \
  } while (0)
  const int nown = (r - rank + P - 1) / P;   // columns rank, rank+P, ...
  for (int j = 0; j < r; ++j) {
    const int par = j & 1;
    double2* col = colbuf + (int64_t)par * d.a;
    if (j % P == rank) {
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
        if (!(bb > 0.0) || !(bb < INFINITY)) set_status(L.status, kStatusSingular);
        if (ib >= r) ib = j;
        s_p = ib;
        stcg(pivbuf + par, ib);
      }
      __syncthreads();
      const int p = s_p;
      for (int i = tid; i < r; i += blockDim.x) {
        int src = i == j ? p : (i == p ? j : i);
        stcg(col + i, X[src + j * ld]);
      }
    }
    BARRIER();
    const int p = ldcg(pivbuf + par);
    if (tid == 0) {
      ipiv[j] = p;
      s_inv = cdiv(mk(1.0, 0.0), ldcg(col + j));
    }
    __syncthreads();
    const double2 inv = s_inv;
    // own columns c != j: exchange rows j, p; scale row j
    for (int q = tid; q < nown; q += blockDim.x) {
      int c = rank + q * P;
      if (c == j) continue;
      double2 xj = X[j + c * ld], xp = X[p + c * ld];
      double2 t = cmul(xp, inv);
      X[j + c * ld] = t;
      if (p != j) X[p + c * ld] = xj;
      tc[q] = t;
    }
    __syncthreads();
    // eliminate column j from the other rows of the own columns
    for (int64_t e = tid; e < (int64_t)nown * r; e += blockDim.x) {
      int q = (int)(e / r), i = (int)(e % r);
      int c = rank + q * P;
      if (c == j || i == j) continue;
      double2 xv = X[i + c * ld];
      cfms(xv, ldcg(col + i), tc[q]);
      X[i + c * ld] = xv;
    }
    if (j % P == rank) {
      for (int i = tid; i < r; i += blockDim.x)
        X[i + j * ld] = i == j ? inv : csub(mk(0.0, 0.0), cmul(ldcg(col + i), inv));
    }
    __syncthreads();
  }
  // undo the row interchanges as a column permutation: final[:, k] = X[:, lab[k]]
  if (tid == 0) {
    for (int k = 0; k < r; ++k) idx[k] = k;
    for (int j = r - 1; j >= 0; --j) {
      int t = idx[j]; idx[j] = idx[ipiv[j]]; idx[ipiv[j]] = t;
    }
  }
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    int c = idx[k];
    if (c % P != rank) continue;
    for (int i = tid; i < r; i += blockDim.x) stcg(Y + i + (int64_t)k * ld, X[i + c * ld]);
  }
  BARRIER();
  for (int q = 0; q < nown; ++q) {
    int c = rank + q * P;
    for (int i = tid; i < r; i += blockDim.x) X[i + c * ld] = ldcg(Y + i + (int64_t)c * ld);
  }
#undef BARRIER
}

size_t gj_dist_scratch_bytes(int a) {
  size_t bytes = 16 + 16 * (2 * (size_t)a + (size_t)a * a);
  return (bytes + 255) & ~(size_t)255;
}

static size_t gj_smem(int amax) { return (size_t)amax * (16 + 4 + 4) + 16; }

int gj_dist_capacity(int amax) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  size_t sm = gj_smem(amax);
  cudaFuncSetAttribute(k_gj_dist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gj_dist, kGjThreads, sm);
  return occ * sms;
}

cudaError_t launch_gj_dist(const LevelDev& L, const CpqrPart* d_parts, int nparts,
                           unsigned char* scratch, int amax, cudaStream_t st) {
  size_t sm = gj_smem(amax);
  cudaError_t e = cudaFuncSetAttribute(k_gj_dist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  LevelDev Lc = L;
  const CpqrPart* pp = d_parts;
  unsigned char* sp = scratch;
  void* args[] = {&Lc, &pp, &sp};
  FMMLU_LAUNCH("xrr_inverse", st,
               e = cudaLaunchCooperativeKernel((const void*)k_gj_dist, dim3(nparts),
                                               dim3(kGjThreads), args, sm, st));
  return e;
}

// ---------------------------------------------------------------------------
// fp32 Gauss-Jordan inverse of X_RR over a thread-block cluster of P CTAs per
// box: the starting point of the Newton-Schulz refinement on the tensor cores.
// Column c lives in the shared memory of CTA c mod P. Per step j, after one
// cluster barrier every CTA reads column j from its owner (distributed shared
// memory), takes the same pivot (largest modulus at or below j, ties to the
// lowest index) and updates its own columns; the owner keeps the new column j
// (the step's coefficients) aside and stores it after the next barrier, when
// no CTA reads it any more. Every CTA runs the same steps, so every cluster
// barrier is reached by all of them. At the end each CTA writes its columns,
// permuted back by the row interchanges, to Xinv as complex128; while loading
// it stores a complex128 copy of X_RR for the refinement.

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ uint32_t cl_map(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ float2 cl_ld(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}

constexpr int kGj32Threads = 256;

size_t gj32_smem(int rmax, int P) {
  const size_t nown = (size_t)(rmax + P - 1) / P;
  return nown * rmax * 8 + 2 * (size_t)rmax * 8 + 2 * (size_t)rmax * 4 + (size_t)nown * 16 + 64;
}

__global__ void __launch_bounds__(kGj32Threads) k_gj32(LevelDev L, int b0,
                                                       const TcUnit* __restrict__ units, int rmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t rank = cl_rank();
  uint32_t csize;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(csize));
  const int Pc = (int)csize;
  const TcUnit u = units[cl_id()];
  const int b = b0 + u.box;
  const BoxDesc& d = L.desc[b];
  const int r = L.run[b].r;
  const int64_t lda = d.a;
  const int nown_max = (rmax + Pc - 1) / Pc;
  float2* cols = reinterpret_cast<float2*>(smem_raw);               // nown_max x rmax
  float2* colj = cols + (size_t)nown_max * rmax;                     // rmax
  float2* pend = colj + rmax;                                         // rmax
  int* ipiv = reinterpret_cast<int*>(pend + rmax);                    // rmax
  int* pos = ipiv + rmax;                                             // rmax
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int nown = r > (int)rank ? (r - (int)rank + Pc - 1) / Pc : 0;
  double2* X = L.arena + d.Xinv_off;
  double2* Acopy = L.nsbuf + L.ns_off[b];
  for (int q = warp; q < nown; q += nw) {
    const int64_t c = (int)rank + q * Pc;
    for (int i = lane; i < r; i += 32) {
      const double2 v = X[i + c * lda];
      Acopy[i + c * lda] = v;
      cols[(size_t)q * r + i] = make_float2((float)v.x, (float)v.y);
    }
  }
  int pend_q = -1;
  cl_sync();
  for (int j = 0; j < r; ++j) {
    if (j > 0) cl_sync();   // column j is final; nobody reads column j-1 any more
    if (pend_q >= 0) {
      for (int i = tid; i < r; i += blockDim.x) cols[(size_t)pend_q * r + i] = pend[i];
      pend_q = -1;
    }
    // column j from its owner
    const int own = j % Pc, qj = j / Pc;
    const uint32_t src =
        cl_map((uint32_t)__cvta_generic_to_shared(cols + (size_t)qj * r), (uint32_t)own);
    for (int i = tid; i < r; i += blockDim.x) colj[i] = cl_ld(src + 8u * (uint32_t)i);
    __syncthreads();
    // every warp finds the same pivot (largest modulus at or below j, ties to
    // the lowest index) on its own: no further CTA-wide synchronisation
    float best = -1.f;
    int bi = r;
    for (int i = j + lane; i < r; i += 32) {
      const float v = colj[i].x * colj[i].x + colj[i].y * colj[i].y;
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    const int p = bi < r ? bi : j;
    const float2 pv = colj[p];
    const float den = pv.x * pv.x + pv.y * pv.y;
    const float2 inv = den > 0.f ? make_float2(pv.x / den, -pv.y / den) : make_float2(0.f, 0.f);
    if (tid == 0) ipiv[j] = p;
    // own columns c != j, one warp per column: t = x_p inv (new row j), x_j to row p
    for (int q = warp; q < nown; q += nw) {
      if ((int)rank + q * Pc == j) continue;
      float2* col = cols + (size_t)q * r;
      const float2 t = cmul(col[p], inv);
      const float2 xj = col[j];
      __syncwarp();
      for (int i = lane; i < r; i += 32) {
        float2 nv;
        if (i == j) nv = t;
        else if (i == p) { nv = xj; cfms(nv, colj[j], t); }
        else { nv = col[i]; cfms(nv, colj[i], t); }
        col[i] = nv;
      }
    }
    if (own == (int)rank) {   // coefficients of step j, stored after the next barrier
      for (int i = tid; i < r; i += blockDim.x) {
        float2 e;
        if (i == j) e = inv;
        else e = cmul(i == p ? colj[j] : colj[i], make_float2(-inv.x, -inv.y));
        pend[i] = e;
      }
      pend_q = qj;
    }
  }
  __syncthreads();
  if (pend_q >= 0)
    for (int i = tid; i < r; i += blockDim.x) cols[(size_t)pend_q * r + i] = pend[i];
  // undo the row interchanges as a column permutation: final[:, k] = X[:, idx[k]]
  if (tid == 0) {
    for (int k = 0; k < r; ++k) pos[k] = k;       // pos holds idx here
    for (int j = r - 1; j >= 0; --j) {
      const int t = pos[j]; pos[j] = pos[ipiv[j]]; pos[ipiv[j]] = t;
    }
    for (int k = 0; k < r; ++k) ipiv[pos[k]] = k; // ipiv now: column c -> position
  }
  __syncthreads();
  for (int q = warp; q < nown; q += nw) {
    const int c = (int)rank + q * Pc;
    double2* dst = X + (int64_t)ipiv[c] * lda;
    for (int i = lane; i < r; i += 32) {
      const float2 v = cols[(size_t)q * r + i];
      dst[i] = make_double2((double)v.x, (double)v.y);
    }
  }
  cl_sync();   // no CTA leaves while another may still read its shared memory
}

int gj32_cluster_size(int rmax) {
  const size_t limit = 227 * 1024;
  for (int P : {8, 16})
    if (gj32_smem(rmax, P) <= limit) return P;
  return 0;
}

cudaError_t launch_gj32(const LevelDev& L, int b0, const TcUnit* d_units, int nunits, int rmax,
                        int P, cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  const size_t sm = gj32_smem(rmax, P);
  cudaError_t e = cudaFuncSetAttribute(k_gj32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  if (P > 8) {
    e = cudaFuncSetAttribute(k_gj32, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nunits * P));
  cfg.blockDim = dim3(kGj32Threads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, k_gj32, &cfg);
  if (e != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return cudaErrorNotSupported;   // the caller inverts these boxes in fp64 instead
  }
  FMMLU_LAUNCH("xrr_inverse32", st, e = cudaLaunchKernelEx(&cfg, k_gj32, L, b0, d_units, rmax));
  return e;
}

}  // namespace fmmlu
