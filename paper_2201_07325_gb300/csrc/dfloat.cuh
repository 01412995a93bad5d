// Double-float arithmetic: a value is the unevaluated sum h + l of two fp32
// numbers (about 46 significant bits). On GB300 the fp32 pipe is 64 times
// wider than the fp64 pipe, and the conversions between fp32 and fp64 share
// the fp64 pipe, so the dot products of the factor apply run here, with the
// conversions done by integer operations on the bit patterns.
//
// Error-free transformations (published methods): Knuth's two-sum for the
// sum of two fp32 numbers, and the FMA residual a*b - fl(a*b) for their
// product. The explicit _rn intrinsics keep the compiler from contracting or
// reassociating them. A dot product accumulated with df_mac is accurate to
// about 2^-46 of the sum of the magnitudes of its terms.
#pragma once

#include <cuda_runtime.h>

namespace fmmlu {

struct DF {
  float h, l;
};

// fp64 -> double-float from the bit pattern, integer operations only: h takes
// the sign, the exponent and the top 23 stored mantissa bits, l the next 23
// (both truncated, so h + l is within 2^-46 |x| of x). Magnitudes below
// 2^-126 give h = 0 and below 2^-80 give l = 0; magnitudes of 2^128 and
// more give an infinite h (NaN stays NaN).
__device__ __forceinline__ DF df_split_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned sgn = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023;
  const unsigned mh = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // stored bits 51 .. 29
  const unsigned ml = (lo >> 6) & 0x7FFFFFu;                  // stored bits 28 .. 6
  float h = 0.f, l = 0.f;
  if (e > 127) {
    const bool nan = e == 1024 && (((hi & 0xFFFFFu) | lo) != 0u);
    h = __uint_as_float(sgn | 0x7F800000u | (nan ? 0x400000u : 0u));
  } else if (e >= -126) {
    h = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | mh);
    if (e >= -80) {
      // ml as an exact fp32 integer (below 2^23) times 2^(e - 46)
      const float mlf = __fsub_rn(__uint_as_float(0x4B000000u | ml), 8388608.0f);
      l = __fmul_rn(mlf, __uint_as_float(sgn | ((unsigned)(e - 46 + 127) << 23)));
    }
  }
  return DF{h, l};
}

// fp32 -> fp64 from the bit pattern (exact for normal numbers, zeros and
// infinities; subnormal fp32 inputs give a signed zero), integer operations
// only: on GB300 the conversion instructions share the narrow fp64 pipe
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned long long sgn = (unsigned long long)(b & 0x80000000u) << 32;
  const unsigned long long ee = e == 255u ? 2047ull : (unsigned long long)(e + 896u);
  const unsigned long long body = (ee << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)(e == 0u ? sgn : (sgn | body)));
}

// double-float -> fp64: one fp64 addition
__device__ __forceinline__ double df_value(DF a) { return f2d_bits(a.h) + f2d_bits(a.l); }

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.h, -a.l}; }

// s += x y
__device__ __forceinline__ void df_mac(DF& s, DF x, DF y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  const float t = __fadd_rn(s.h, p);
  const float bp = __fsub_rn(t, s.h);
  const float err = __fadd_rn(__fsub_rn(s.h, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s.l = __fadd_rn(s.l, __fadd_rn(err, e));
  s.h = t;
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float t = __fadd_rn(a.h, b.h);
  const float bp = __fsub_rn(t, a.h);
  const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(t, bp)), __fsub_rn(b.h, bp));
  return DF{t, __fadd_rn(err, __fadd_rn(a.l, b.l))};
}

// complex double-float, stored as float4 {re.h, re.l, im.h, im.l}
__device__ __forceinline__ float4 cdf_split_bits(double2 v) {
  const DF r = df_split_bits(v.x), i = df_split_bits(v.y);
  return make_float4(r.h, r.l, i.h, i.l);
}

// (re, im) += op(m) x, op = conj when kCj
template <bool kCj>
__device__ __forceinline__ void cdf_mac(DF& re, DF& im, DF mr, DF mi, float4 x) {
  const DF xr{x.x, x.y}, xi{x.z, x.w};
  df_mac(re, mr, xr);
  df_mac(im, mr, xi);
  if (kCj) {
    df_mac(re, mi, xi);
    df_mac(im, df_neg(mi), xr);
  } else {
    df_mac(re, df_neg(mi), xi);
    df_mac(im, mi, xr);
  }
}

// sum of a DF over the `w` lanes of an aligned lane group (w a power of two)
__device__ __forceinline__ DF df_group_sum(DF v, int w) {
  for (int o = w >> 1; o > 0; o >>= 1) {
    const DF u{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
    v = df_add(v, u);
  }
  return v;
}

}  // namespace fmmlu
