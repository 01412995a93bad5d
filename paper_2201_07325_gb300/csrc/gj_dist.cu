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

}  // namespace fmmlu
