// Device helpers: complex arithmetic and the Helmholtz kernel evaluations.
//
// Kernel definitions (Sec. 3):
//   G(x, y) = exp(i k r) / (4 pi r),  r = |x - y|            (Eq. greenfunhelm)
//   K(x, y) = n(y) . grad_y G(x, y) - i eta G(x, y)            (Eq. comb_ref)
//   n(y) . grad_y G = G (i k r - 1) / r^2 ((y - x) . n(y))
//   A_ij = sqrt(w_i) K(x_i, x_j) sqrt(w_j) (i != j),
//   A_ii = 1/2 - i eta (sqrt(w_i/pi)/2 + i k w_i/(4 pi))       (Eq. disc3)
// The transcendental functions are CUDA's own (sincos, sqrt, division).
#pragma once

#include <cuda_runtime.h>
#include "fmmlu_internal.h"

namespace fmmlu {

template <typename R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return mk(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return mk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
__host__ __device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__host__ __device__ __forceinline__ void cfma_cj(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
// acc -= a * b (four fused multiply-adds)
__host__ __device__ __forceinline__ void cfms(double2& acc, double2 a, double2 b) {
  acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
// acc += |a|^2 (two fused multiply-adds)
__host__ __device__ __forceinline__ void cnorm_acc(double& acc, double2 a) {
  acc = fma(a.x, a.x, acc); acc = fma(a.y, a.y, acc);
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return mk((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return mk(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return mk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ void cfma_cj(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ void cfms(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(-a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(-a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ void cnorm_acc(float& acc, float2 a) {
  acc = fmaf(a.x, a.x, acc); acc = fmaf(a.y, a.y, acc);
}
__host__ __device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
  float d = b.x * b.x + b.y * b.y;
  return mk((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
template <typename C> __device__ __forceinline__ C from_d2(double2 a);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

// G(t, s) = exp(i k r)/(4 pi r)
__device__ __forceinline__ double2 green(double tx, double ty, double tz, double sx,
                                         double sy, double sz, double k) {
  double dx = sx - tx, dy = sy - ty, dz = sz - tz;
  double r = sqrt(dx * dx + dy * dy + dz * dz);
  double sn, cs;
  sincos(k * r, &sn, &cs);
  double g = 1.0 / (4.0 * kPi * r);
  return mk(cs * g, sn * g);
}

// K(t, s) = n(s).grad_s G(t, s) - i eta G(t, s)
__device__ __forceinline__ double2 comb_kernel(double tx, double ty, double tz,
                                               double sx, double sy, double sz,
                                               double nx, double ny, double nz,
                                               double k, double eta) {
  double dx = sx - tx, dy = sy - ty, dz = sz - tz;
  double r2 = dx * dx + dy * dy + dz * dz;
  double r = sqrt(r2);
  double sn, cs;
  sincos(k * r, &sn, &cs);
  double ginv = 1.0 / (4.0 * kPi * r);
  double2 g = mk(cs * ginv, sn * ginv);
  double proj = (dx * nx + dy * ny + dz * nz) / r2;   // ((s - t).n(s)) / r^2
  // (i k r - 1) * proj
  double2 f = mk(-proj, k * r * proj);
  double2 d = cmul(g, f);
  // - i eta g = (eta g.y, -eta g.x)
  return mk(d.x + eta * g.y, d.y - eta * g.x);
}

// Single-precision versions for the mixed path's ID matrix: the coordinate
// differences are formed in fp64 (cancellation), everything after in fp32
// with CUDA's fp32 sincos and square root.
__device__ __forceinline__ float2 green_f(double tx, double ty, double tz, double sx, double sy,
                                         double sz, float k) {
  float dx = (float)(sx - tx), dy = (float)(sy - ty), dz = (float)(sz - tz);
  float r = sqrtf(dx * dx + dy * dy + dz * dz);
  float sn, cs;
  sincosf(k * r, &sn, &cs);
  float g = 1.0f / (4.0f * (float)kPi * r);
  return make_float2(cs * g, sn * g);
}

__device__ __forceinline__ float2 comb_kernel_f(double tx, double ty, double tz, double sx,
                                               double sy, double sz, float nx, float ny,
                                               float nz, float k, float eta) {
  float dx = (float)(sx - tx), dy = (float)(sy - ty), dz = (float)(sz - tz);
  float r2 = dx * dx + dy * dy + dz * dz;
  float r = sqrtf(r2);
  float sn, cs;
  sincosf(k * r, &sn, &cs);
  float ginv = 1.0f / (4.0f * (float)kPi * r);
  float2 g = make_float2(cs * ginv, sn * ginv);
  float proj = (dx * nx + dy * ny + dz * nz) / r2;
  float2 f = make_float2(-proj, k * r * proj);
  float2 d = cmul(g, f);
  return make_float2(d.x + eta * g.y, d.y - eta * g.x);
}

// Matrix entry A(i, j) of the scaled system without Schur updates.
__device__ __forceinline__ double2 entry(const Geometry& g, int i, int j) {
  if (i == j) {
    double w = g.w[i];
    return mk(0.5 + g.eta * g.k * w / (4.0 * kPi), -g.eta * sqrt(w / kPi) * 0.5);
  }
  double2 kv = comb_kernel(g.px[i], g.py[i], g.pz[i], g.px[j], g.py[j], g.pz[j],
                           g.nx[j], g.ny[j], g.nz[j], g.k, g.eta);
  return cscale(kv, g.sw[i] * g.sw[j]);
}

// K(t, s) and K(s, t) of one pair from a single evaluation of G(t, s) = G(s, t):
//   K(t, s) = G (i k r - 1) ((s - t).n(s)) / r^2 - i eta G
//   K(s, t) = G (i k r - 1) ((t - s).n(t)) / r^2 - i eta G
template <typename R>
__device__ __forceinline__ void comb_kernel_pair(R dx, R dy, R dz,   // s - t
                                                 R tnx, R tny, R tnz, R snx, R sny, R snz, R k,
                                                 R eta, typename CT<R>::T& kts,
                                                 typename CT<R>::T& kst, typename CT<R>::T& g) {
  const R r2 = dx * dx + dy * dy + dz * dz;
  const R r = sqrt(r2);
  const R inv_r2 = R(1) / r2;     // the one division: 1/r = r / r^2
  R sn, cs;
  sincos(k * r, &sn, &cs);
  const R ginv = (r * inv_r2) * R(1.0 / (4.0 * kPi));
  g = mk(cs * ginv, sn * ginv);
  const typename CT<R>::T gf = cmul(g, mk(R(-1), k * r));   // G (i k r - 1)
  const R pts = (dx * snx + dy * sny + dz * snz) * inv_r2;
  const R pst = -(dx * tnx + dy * tny + dz * tnz) * inv_r2;
  kts = mk(gf.x * pts + eta * g.y, gf.y * pts - eta * g.x);
  kst = mk(gf.x * pst + eta * g.y, gf.y * pst - eta * g.x);
}

// A(i, j) and A(j, i) of the scaled system (i != j), one kernel evaluation
__device__ __forceinline__ void entry_pair(const Geometry& g, int i, int j, double2& aij,
                                           double2& aji) {
  if (i == j) {
    aij = aji = entry(g, i, i);
    return;
  }
  double2 kij, kji, gg;
  comb_kernel_pair<double>(g.px[j] - g.px[i], g.py[j] - g.py[i], g.pz[j] - g.pz[i], g.nx[i],
                           g.ny[i], g.nz[i], g.nx[j], g.ny[j], g.nz[j], g.k, g.eta, kij, kji, gg);
  const double sc = g.sw[i] * g.sw[j];
  aij = cscale(kij, sc);
  aji = cscale(kji, sc);
}

// one coordinate of s - t from the split fp32 copies: the high parts'
// difference is rounded once, the low parts restore what rounding each
// coordinate to fp32 dropped
__device__ __forceinline__ float fdiff(const float* h, const float* l, int s, int t) {
  return (h[s] - h[t]) + (l[s] - l[t]);
}

// A(i, j) and A(j, i) of the scaled system (i != j), one kernel evaluation in
// fp32 (CUDA's fp32 sincos and square root) from the split copies
__device__ __forceinline__ void entry_pair_f(const GeometryF& f, float k, float eta, int i, int j,
                                             float2& aij, float2& aji) {
  float2 kij, kji, gg;
  comb_kernel_pair<float>(fdiff(f.xh, f.xl, j, i), fdiff(f.yh, f.yl, j, i),
                          fdiff(f.zh, f.zl, j, i), f.nx[i], f.ny[i], f.nz[i], f.nx[j], f.ny[j],
                          f.nz[j], k, eta, kij, kji, gg);
  const float sc = f.sw[i] * f.sw[j];
  aij = cscale(kij, sc);
  aji = cscale(kji, sc);
}

// l-th of n Fibonacci points on the unit sphere
__device__ __forceinline__ void fib_point(int l, int n, double& ux, double& uy,
                                          double& uz) {
  double z = 1.0 - (2.0 * l + 1.0) / n;
  double phi = l * kGoldenAngle;
  double rho = sqrt(fmax(0.0, 1.0 - z * z));
  double sn, cs;
  sincos(phi, &sn, &cs);
  ux = rho * cs; uy = rho * sn; uz = z;
}

__device__ __forceinline__ void set_status(int* status, int bits) {
  if (status) atomicOr(status, bits);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace fmmlu
