// Monostatic sonar cross section (Sec. 6.3): incident plane waves and the
// backscattered far field of the combined-field layer potential.
//
// For a plane wave exp(i k d.x) travelling along the unit direction d the
// sound-soft boundary data are f = -exp(i k d.x), so b_j = -sqrt(w_j)
// exp(i k d.x_j). With the density x~ = sqrt(w) sigma of the solved system,
// u(t) = sum_j K(t, x_j) sqrt(w_j) x~_j and, as |t| -> infinity along the
// unit vector t^, K(t, y) ~ exp(i k |t|)/(4 pi |t|) exp(-i k t^.y)
// (-i k n(y).t^ - i eta). The monostatic (backscattered, t^ = -d) far-field
// pattern is therefore
//   R(d) = (1/(4 pi)) sum_j sqrt(w_j) x~_j exp(i k d.x_j) (i k n_j.d - i eta)
//        = (-i k / (4 pi)) sum_j sqrt(w_j) x~_j exp(i k d.x_j) (1 - n_j.d)   (eta = k).
// Sums over the points run as per-block partial sums added in a fixed order.
#include <algorithm>

#include "device_common.cuh"

namespace fmmlu {

constexpr int kSonThreads = 256;

// b[j + m n] = -sqrt(w_j) exp(i k d_m . x_j)
__global__ void k_plane_waves(const double* __restrict__ pts, const double* __restrict__ w,
                              int64_t n, double k, const double* __restrict__ dirs, int m0,
                              double2* __restrict__ b) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int m = m0 + blockIdx.y;
  if (j >= n) return;
  const double* d = dirs + 3 * m;
  const double ph = k * (d[0] * pts[3 * j] + d[1] * pts[3 * j + 1] + d[2] * pts[3 * j + 2]);
  double sn, cs;
  sincos(ph, &sn, &cs);
  const double s = -sqrt(w[j]);
  b[j + (int64_t)blockIdx.y * n] = mk(s * cs, s * sn);
}

// part[blk + nblk m] = partial sum over the block's rows of
// sqrt(w_j) x~_{j,m} exp(i k d_m . x_j) (i k n_j.d_m - i eta)
__global__ void __launch_bounds__(kSonThreads)
    k_backscatter_partial(const double* __restrict__ pts, const double* __restrict__ nrm,
                          const double* __restrict__ w, int64_t n, double k, double eta,
                          const double* __restrict__ dirs, int m0,
                          const double2* __restrict__ x, int64_t rows_per_blk,
                          double2* __restrict__ part) {
  __shared__ double2 red[kSonThreads / 32];
  const int m = m0 + blockIdx.y;
  const double* d = dirs + 3 * m;
  const double2* xc = x + (int64_t)blockIdx.y * n;
  const int64_t i0 = blockIdx.x * rows_per_blk, i1 = min(n, i0 + rows_per_blk);
  double2 acc = mk(0.0, 0.0);
  for (int64_t j = i0 + threadIdx.x; j < i1; j += blockDim.x) {
    const double px = pts[3 * j], py = pts[3 * j + 1], pz = pts[3 * j + 2];
    const double nd = nrm[3 * j] * d[0] + nrm[3 * j + 1] * d[1] + nrm[3 * j + 2] * d[2];
    double sn, cs;
    sincos(k * (d[0] * px + d[1] * py + d[2] * pz), &sn, &cs);
    // exp(i k d.x) (i (k n.d - eta)) sqrt(w)
    const double c = (k * nd - eta) * sqrt(w[j]);
    const double2 f = mk(-sn * c, cs * c);
    cfma(acc, f, xc[j]);
  }
  acc.x = warp_sum(acc.x);
  acc.y = warp_sum(acc.y);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = red[0];
    for (int q = 1; q < kSonThreads / 32; ++q) s = cadd(s, red[q]);
    part[blockIdx.x + (int64_t)gridDim.x * blockIdx.y] = s;
  }
}

__global__ void k_backscatter_final(const double2* __restrict__ part, int nblk, int mcount,
                                    int m0, double2* __restrict__ R) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= mcount) return;
  double2 s = mk(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) s = cadd(s, part[b + (int64_t)nblk * m]);
  R[m0 + m] = cscale(s, 1.0 / (4.0 * kPi));
}

static int64_t son_rows_per_block(int64_t n) { return std::max<int64_t>(8192, (n + 511) / 512); }

int backscatter_blocks(int64_t n) {
  const int64_t r = son_rows_per_block(n);
  return (int)((n + r - 1) / r);
}

void launch_plane_waves(const double* pts, const double* w, int64_t n, double k,
                        const double* dirs, int m0, int mcount, double2* b, cudaStream_t st) {
  if (mcount <= 0) return;
  dim3 grid((unsigned)((n + kSonThreads - 1) / kSonThreads), (unsigned)mcount);
  FMMLU_LAUNCH("plane_waves", st,
               k_plane_waves<<<grid, kSonThreads, 0, st>>>(pts, w, n, k, dirs, m0, b));
}

void launch_backscatter(const double* pts, const double* nrm, const double* w, int64_t n,
                        double k, double eta, const double* dirs, int m0, int mcount,
                        const double2* x, double2* part, double2* R, cudaStream_t st) {
  if (mcount <= 0) return;
  const int64_t rpb = son_rows_per_block(n);
  const int nblk = backscatter_blocks(n);
  FMMLU_LAUNCH("backscatter", st,
               k_backscatter_partial<<<dim3(nblk, mcount), kSonThreads, 0, st>>>(
                   pts, nrm, w, n, k, eta, dirs, m0, x, rpb, part));
  FMMLU_LAUNCH("backscatter", st,
               k_backscatter_final<<<(mcount + 127) / 128, 128, 0, st>>>(part, nblk, mcount, m0,
                                                                         R));
}

}  // namespace fmmlu
