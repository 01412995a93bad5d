// Exactly split complex products on the fifth-generation tensor cores
// (tcgen05.mma with accumulators in tensor memory, operands staged by bulk
// copies).
//
// C = op(A) B (A m x k, B k x n, complex128 or complex64; op = identity or
// conjugation) is formed as follows. Every row of A and every column of B is
// scaled by a power of two 2^e taken from its largest component and written as
// NS balanced base-256 digits c_0 .. c_{NS-1} in [-128, 128], exact in bf16:
//     v ~ 2^e sum_p c_p 2^{-8(p+1)}        (the leading 8 NS - 1 bits of v/2^e).
// Then C_ij = 2^{e_i + e_j - 16} sum_{d <= DMAX} 2^{-8d} S_d(i, j), where S_d is
// the integer matrix sum_{p+q=d} op(A_p) B_q. Each S_d has its own fp32
// accumulator in tensor memory; it is read out (into 64-bit integers) after a
// window of W_d k16-steps with W_d (pairs in the group) <= 32, so every partial
// sum is an integer of magnitude <= 2^24 and exact in fp32. The only rounding is
// the final conversion of the integers to double.
//
// One CTA computes a 128 x 32 complex tile. A complex product is two MMAs of
// N = 64: B is staged as three 32-row parts, [-Bi | Br | Bi] (or [Br | Bi | -Br]
// for conj(A)), so that A_re x [Br ; Bi] + A_im x [-Bi ; Br] = [Cr | Ci].
// Warp roles: warp 0 issues the bulk copies of the two-stage operand pipeline,
// warp 1 owns tensor memory and issues the MMAs (one thread), warps 2..9 drain
// the accumulators (warp w reads tensor-memory lanes 32 (w % 4) .. + 31).
// Every wait is bounded; on a timeout the CTA records kStatusTimeout, lets its
// copies and MMAs in flight finish (bounded), frees tensor memory and returns.
//
// Global layouts written by the split kernels (both per box, k in steps of 16):
//   A: [row block of 128][k16 step][digit p][part re, im][128 x 16 bf16]
//   B: [column block of 32][k16 step][digit q][96 x 16 bf16 (three parts)]
// where a 128 x 16 (96 x 16) block is in the K-major core-matrix order of the
// MMA's shared-memory descriptor: 8 x 8 core matrices of 128 contiguous bytes,
// row groups 128 B apart, the two k halves 2048 B (1536 B) apart.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "device_common.cuh"
#include "dfloat.cuh"

namespace fmmlu {

namespace tc {

constexpr int kThreads = 320;
constexpr int kRows = 128;                      // tile rows (MMA M)
constexpr int kCols = 32;                       // complex tile columns (MMA N = 64)
constexpr int kAChunk = kRows * 16 * 2;         // one digit part of A, one k16 step
// 8-row groups stored per k-half of an A chunk: an operand with at most 128
// rows keeps only its own rows (the MMA still reads 128; the rows past the
// operand hold other data and give output rows that are never stored)
__host__ __device__ __forceinline__ int a_groups(int m) { return m <= kRows ? (m + 7) / 8 : kRows / 8; }
__host__ __device__ __forceinline__ int a_chunk(int m) { return a_groups(m) * 256; }
constexpr int kBChunk = 3 * kCols * 16 * 2;     // one digit of B (three parts)
constexpr long long kWaitLimit = 20000000;      // polls (~1-2 s)

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(c) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try(uint64_t* b, uint32_t par) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(par)
      : "memory");
  return ok;
}
// bounded wait; false on timeout or when another thread of the CTA gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t par, volatile int* abort_flag) {
  for (long long i = 0; i < kWaitLimit; ++i) {
    if (mbar_try(b, par)) return true;
    if ((i & 1023) == 1023 && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(b))
      : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of tcgen05
  return d;
}
// instruction descriptor of kind::f16: bf16 A and B (K-major), fp32 D
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc(kRows, 2 * kCols)), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void commit(uint64_t* b) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (r, k) in a rows x 16 block in core-matrix order
__device__ __forceinline__ int canon16(int r, int k, int rows) {
  return ((k >> 3) * (rows >> 3) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// digit pairs of group d and window lengths (k16 steps)
__host__ __device__ constexpr int plo(int d, int ns) { return d > ns - 1 ? d - (ns - 1) : 0; }
__host__ __device__ constexpr int phi(int d, int ns) { return d < ns - 1 ? d : ns - 1; }
__host__ __device__ constexpr int window(int d, int ns) { return 32 / (phi(d, ns) - plo(d, ns) + 1); }

// balanced base-256 digits of v / 2^e (|v| < 2^(e-1)): NS of them, c_0 first,
// c_p in [-128, 128]. |v| 2^(8 NS - e) truncated toward zero is read off the
// bits of v (integer shifts of the significand, no fp64 arithmetic); its bytes
// are balanced by carrying into the next byte up; the sign is applied last.
template <int NS>
__device__ __forceinline__ void balanced_digits(double v, int e, int* c) {
  static_assert(NS == 4 || NS == 7, "digit counts of the complex64 / complex128 splits");
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const bool neg = (u >> 63) != 0;
  const int E = (int)((u >> 52) & 0x7FF);
  unsigned long long mant = u & 0xFFFFFFFFFFFFFull;
  int ex = -1074;                          // zero or subnormal: mant 2^-1074
  if (E != 0) { mant |= 1ull << 52; ex = E - 1075; }
  const int sh = ex + 8 * NS - e;          // |v| 2^(8 NS - e) = mant 2^sh < 2^(8 NS - 1)
  const unsigned long long U = sh >= 0 ? mant << sh : (sh > -64 ? mant >> (-sh) : 0ull);
  const uint32_t lo = (uint32_t)U, hi = (uint32_t)(U >> 32);
  int carry = 0;
#pragma unroll
  for (int i = NS - 1; i >= 1; --i) {
    const int byte_index = NS - 1 - i;     // byte of U, least significant first
    const uint32_t word = byte_index < 4 ? lo : hi;
    int dg = (int)((word >> (8 * (byte_index & 3))) & 255u) + carry;
    carry = dg >= 128 ? 1 : 0;
    c[i] = dg - 256 * carry;
  }
  {
    const int byte_index = NS - 1;
    const uint32_t word = byte_index < 4 ? lo : hi;
    c[0] = (int)((word >> (8 * (byte_index & 3))) & 255u) + carry;   // <= 128
  }
  if (neg) {
#pragma unroll
    for (int i = 0; i < NS; ++i) c[i] = -c[i];
  }
}

// two small integers (|c| <= 128) as a packed bf16 pair, exactly: the fp32
// value of c has at most 8 significant bits, so its upper half is its bf16
__device__ __forceinline__ uint32_t bf16_pair(int lo, int hi) {
  const float fl = __int_as_float(0x4B400000 + lo) - 12582912.0f;
  const float fh = __int_as_float(0x4B400000 + hi) - 12582912.0f;
  return __byte_perm(__float_as_uint(fl), __float_as_uint(fh), 0x7632);
}

}  // namespace tc

// ---------------------------------------------------------------------------
// problems: sizes of one box, element accessors of op-free A (m x k) and
// B (k x n), and the epilogue

struct TcExtra {
  const GramBoxHost* gb;
  double2* gbuf;
  // split-K products: per box (descriptor index) the offset of its int64
  // accumulator (4 per entry: hi re, hi im, lo re, lo im)
  unsigned long long* gx;
  const int64_t* gx_off;
};

// k16 steps per chunk of a split-K problem (0: no split)
template <class Prob> struct TcSplit { static constexpr int steps = 0; };

// kAk / kBk: consecutive k of one row of A / column of B are contiguous in memory
struct TcSchur {    // Delta(S|N, S|N) -= W X_RC: (s+n) x (s+n) x r
  static constexpr bool kConj = false, kUpper = false, kAk = false, kBk = true;
  __device__ static bool dims(const LevelDev&, const BoxDesc&, const BoxRun& rr, int& m, int& n,
                              int& k) {
    m = rr.s + rr.n; n = m; k = rr.r; return rr.r >= kTcInnerMin;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun&, int i, int kk) {
    return L.Wbuf[d.W_off + i + (int64_t)kk * (d.a + d.nmax)];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, int kk, int j) {
    return L.arena[d.G1_off + rr.s + kk + (int64_t)j * d.a];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, const TcExtra&,
                             int i, int j, double vr, double vi) {
    const int s = rr.s;
    const int* perm = L.iarena + d.idx_off + d.a + d.nmax;
    const int* ndof = L.rows + d.rows_off + 3 * d.qmax;
    const int* npos = ndof + d.nmax;
    const int* nloc = npos + d.nmax;
    const int xl = i < s ? 0 : nloc[i - s], xp = i < s ? perm[i] : npos[i - s];
    const int yl = j < s ? 0 : nloc[j - s], yp = j < s ? perm[j] : npos[j - s];
    const int cnt = 1 + d.ncnt;
    const int64_t off = L.pairtab[d.pairtab + (int64_t)xl * cnt + yl];
    if (off < 0) { set_status(L.status, kStatusBound); return; }
    const int ld = xl == 0 ? d.a : L.cur_a0[L.nlist[d.nbeg + xl - 1]];
    double2* pz = L.delta + off + xp + (int64_t)yp * ld;
    const double2 c = *pz;
    *pz = make_double2(c.x - vr, c.y - vi);
  }
  // The same update split into a per-row part, computed once for a row's 16
  // outputs, and a per-column part; the index arrays are read through the
  // read-only path (nothing writes them during the product), so the
  // compiler may keep and reorder those loads across the pool stores.
  struct Row {
    const int* perm;
    const int* npos;
    const int* nloc;
    int64_t prow;   // pairtab entry of (row's owner, 0)
    int s, xp, ld;
  };
  __device__ static Row row(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, int i) {
    Row w;
    w.s = rr.s;
    w.perm = L.iarena + d.idx_off + d.a + d.nmax;
    const int* ndof = L.rows + d.rows_off + 3 * d.qmax;
    w.npos = ndof + d.nmax;
    w.nloc = w.npos + d.nmax;
    const int xl = i < w.s ? 0 : __ldg(w.nloc + i - w.s);
    w.xp = i < w.s ? __ldg(w.perm + i) : __ldg(w.npos + i - w.s);
    w.prow = d.pairtab + (int64_t)xl * (1 + d.ncnt);
    w.ld = xl == 0 ? d.a : __ldg(L.cur_a0 + __ldg(L.nlist + d.nbeg + xl - 1));
    return w;
  }
  __device__ static void col(const LevelDev& L, const Row& w, int j, double vr, double vi) {
    const int yl = j < w.s ? 0 : __ldg(w.nloc + j - w.s);
    const int yp = j < w.s ? __ldg(w.perm + j) : __ldg(w.npos + j - w.s);
    const int64_t off = __ldg(L.pairtab + w.prow + yl);
    if (off < 0) { set_status(L.status, kStatusBound); return; }
    double2* pz = L.delta + off + w.xp + (int64_t)yp * w.ld;
    const double2 c = *pz;
    *pz = make_double2(c.x - vr, c.y - vi);
  }
};

struct TcNoRow { struct Row {}; };
template <class Prob, class = void> struct TcRowEpi { static constexpr bool value = false; };
template <class Prob>
struct TcRowEpi<Prob, std::void_t<typename Prob::Row>> { static constexpr bool value = true; };

struct TcW {        // W = X_CR X_RR^{-1}: (s+n) x r x r, stored
  static constexpr bool kConj = false, kUpper = false, kAk = false, kBk = true;
  __device__ static bool dims(const LevelDev&, const BoxDesc&, const BoxRun& rr, int& m, int& n,
                              int& k) {
    m = rr.s + rr.n; n = rr.r; k = rr.r; return rr.r >= kTcInnerMin;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, int i, int kk) {
    return L.arena[d.G3_off + i + (int64_t)(rr.s + kk) * (d.a + d.nmax)];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun&, int kk, int j) {
    return L.arena[d.Xinv_off + kk + (int64_t)j * d.a];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun&, const TcExtra&,
                             int i, int j, double vr, double vi) {
    L.Wbuf[d.W_off + i + (int64_t)j * (d.a + d.nmax)] = make_double2(vr, vi);
  }
};

struct TcG1 {       // G1[s:a, :] -= T^T G1[0:s, :]: r x (a+n) x s
  static constexpr bool kConj = false, kUpper = false, kAk = true, kBk = true;
  __device__ static bool dims(const LevelDev&, const BoxDesc& d, const BoxRun& rr, int& m, int& n,
                              int& k) {
    m = rr.r; n = d.a + rr.n; k = rr.s; return rr.r > 0 && rr.s >= kTcInnerMin;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun&, int i, int kk) {
    return L.arena[d.T_off + kk + (int64_t)i * d.a];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun&, int kk, int j) {
    return L.arena[d.G1_off + kk + (int64_t)j * d.a];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, const TcExtra&,
                             int i, int j, double vr, double vi) {
    double2* c = L.arena + d.G1_off + (rr.s + i) + (int64_t)j * d.a;
    const double2 t = *c;
    *c = make_double2(t.x - vr, t.y - vi);
  }
  // per-row part of the update (the row's base and stride), once per 16 outputs
  struct Row {
    double2* base;
    int64_t ld;
  };
  __device__ static Row row(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, int i) {
    return Row{L.arena + d.G1_off + (rr.s + i), (int64_t)d.a};
  }
  __device__ static void col(const LevelDev&, const Row& w, int j, double vr, double vi) {
    double2* c = w.base + (int64_t)j * w.ld;
    const double2 t = *c;
    *c = make_double2(t.x - vr, t.y - vi);
  }
};

struct TcG3 {       // G3[:, s:a] -= G3[:, 0:s] T: (a+n) x r x s
  static constexpr bool kConj = false, kUpper = false, kAk = false, kBk = true;
  __device__ static bool dims(const LevelDev&, const BoxDesc& d, const BoxRun& rr, int& m, int& n,
                              int& k) {
    m = d.a + rr.n; n = rr.r; k = rr.s; return rr.r > 0 && rr.s >= kTcInnerMin;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun&, int i, int kk) {
    return L.arena[d.G3_off + i + (int64_t)kk * (d.a + d.nmax)];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun&, int kk, int j) {
    return L.arena[d.T_off + kk + (int64_t)j * d.a];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, const TcExtra&,
                             int i, int j, double vr, double vi) {
    double2* c = L.arena + d.G3_off + i + (int64_t)(rr.s + j) * (d.a + d.nmax);
    const double2 t = *c;
    *c = make_double2(t.x - vr, t.y - vi);
  }
  // per-row part of the update (the row's base and stride), once per 16 outputs
  struct Row {
    double2* base;
    int64_t ld;
  };
  __device__ static Row row(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, int i) {
    const int64_t ld = d.a + d.nmax;
    return Row{L.arena + d.G3_off + i + (int64_t)rr.s * ld, ld};
  }
  __device__ static void col(const LevelDev&, const Row& w, int j, double vr, double vi) {
    double2* c = w.base + (int64_t)j * w.ld;
    const double2 t = *c;
    *c = make_double2(t.x - vr, t.y - vi);
  }
};

struct TcXrr {      // X_RR = A_RR - A_RS T (before inversion): r x r x s
  static constexpr bool kConj = false, kUpper = false, kAk = false, kBk = true;
  __device__ static bool dims(const LevelDev&, const BoxDesc&, const BoxRun& rr, int& m, int& n,
                              int& k) {
    m = rr.r; n = rr.r; k = rr.s; return rr.r > 0 && rr.s >= kTcInnerMin;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, int i, int kk) {
    return L.arena[d.G1_off + rr.s + i + (int64_t)kk * d.a];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun&, int kk, int j) {
    return L.arena[d.T_off + kk + (int64_t)j * d.a];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, const TcExtra&,
                             int i, int j, double vr, double vi) {
    const double2 y = L.arena[d.G1_off + rr.s + i + (int64_t)(rr.s + rr.n + j) * d.a];
    L.arena[d.Xinv_off + i + (int64_t)j * d.a] = make_double2(y.x - vr, y.y - vi);
  }
};

// Newton-Schulz refinement of X ~ X_RR^{-1} (boxes kNsMin <= r <= ns_rmax):
// Y = X_RR X into the box's product scratch (recording max |I - Y|), then
// X <- 2 X - X Y in place (the operands were split before the product runs).
__device__ __forceinline__ bool ns_box(const LevelDev& L, const BoxDesc& d, const BoxRun& rr) {
  if (rr.r < kNsMin || rr.r > L.ns_rmax) return false;
  return !(L.ns_skip && L.ns_skip[&d - L.desc]);   // a step the box no longer needs
}
struct TcNsY {
  static constexpr bool kConj = false, kUpper = false, kAk = false, kBk = true;
  __device__ static bool dims(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, int& m, int& n,
                              int& k) {
    m = rr.r; n = rr.r; k = rr.r; return ns_box(L, d, rr);
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun&, int i, int kk) {
    const int b = (int)(&d - L.desc);
    return L.nsbuf[L.ns_off[b] + i + (int64_t)kk * d.a];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun&, int kk, int j) {
    return L.arena[d.Xinv_off + kk + (int64_t)j * d.a];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun&, const TcExtra&,
                             int i, int j, double vr, double vi) {
    const int b = (int)(&d - L.desc);
    const int64_t a = d.a;
    L.nsbuf[L.ns_off[b] + a * a + i + j * a] = make_double2(vr, vi);
    const double e = fmax(fabs(vr - (i == j ? 1.0 : 0.0)), fabs(vi));
    atomicMax(&L.ns_err[b], (unsigned long long)__double_as_longlong(e));
  }
};
struct TcNsX {
  static constexpr bool kConj = false, kUpper = false, kAk = false, kBk = true;
  __device__ static bool dims(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, int& m, int& n,
                              int& k) {
    m = rr.r; n = rr.r; k = rr.r; return ns_box(L, d, rr);
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun&, int i, int kk) {
    return L.arena[d.Xinv_off + i + (int64_t)kk * d.a];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun&, int kk, int j) {
    const int b = (int)(&d - L.desc);
    const int64_t a = d.a;
    return L.nsbuf[L.ns_off[b] + a * a + kk + (int64_t)j * a];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun&, const TcExtra&,
                             int i, int j, double vr, double vi) {
    double2* x = L.arena + d.Xinv_off + i + (int64_t)j * d.a;
    const double2 o = *x;
    *x = make_double2(2.0 * o.x - vr, 2.0 * o.y - vi);
  }
};

// Root block elimination, step [i0, i1 = i0 + r), later = n0 - i1:
// W = A[later, i0:i1] D^{-1} (D^{-1} in the diagonal block), then
// A[later, later] -= W A[i0:i1, later]. The level and box arguments are unused.
struct TcRootW {
  static constexpr bool kConj = false, kUpper = false, kAk = false, kBk = true;
  __device__ static bool dims(const LevelDev& L, const BoxDesc&, const BoxRun&, int& m, int& n,
                              int& k) {
    m = (int)(L.root_n0 - L.root_i0 - L.root_r); n = L.root_r; k = L.root_r;
    return m > 0 && k >= kTcInnerMin;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc&, const BoxRun&, int i, int kk) {
    return L.root_A[(L.root_i0 + L.root_r + i) + (int64_t)(L.root_i0 + kk) * L.root_n0];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc&, const BoxRun&, int kk, int j) {
    return L.root_A[(L.root_i0 + kk) + (int64_t)(L.root_i0 + j) * L.root_n0];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc&, const BoxRun&, const TcExtra&,
                             int i, int j, double vr, double vi) {
    const int64_t later = L.root_n0 - L.root_i0 - L.root_r;
    L.root_W[i + j * later] = make_double2(vr, vi);
  }
};
struct TcRootS {
  static constexpr bool kConj = false, kUpper = false, kAk = false, kBk = true;
  __device__ static bool dims(const LevelDev& L, const BoxDesc&, const BoxRun&, int& m, int& n,
                              int& k) {
    m = (int)(L.root_n0 - L.root_i0 - L.root_r); n = m; k = L.root_r;
    return m > 0 && k >= kTcInnerMin;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc&, const BoxRun&, int i, int kk) {
    const int64_t later = L.root_n0 - L.root_i0 - L.root_r;
    return L.root_W[i + kk * later];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc&, const BoxRun&, int kk, int j) {
    return L.root_A[(L.root_i0 + kk) + (int64_t)(L.root_i0 + L.root_r + j) * L.root_n0];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc&, const BoxRun&, const TcExtra&,
                             int i, int j, double vr, double vi) {
    const int64_t i1 = L.root_i0 + L.root_r;
    double2* x = L.root_A + (i1 + i) + (i1 + j) * L.root_n0;
    const double2 o = *x;
    *x = make_double2(o.x - vr, o.y - vi);
  }
};

// The C products of the solve sweeps (Sec. 4.2, factored form of A^{-1}) for
// one colour of the solve plan, all right-hand sides at once. The box is the
// index of the placeholder descriptor d in L.desc, which is also its index in
// L.sbox. Forward: b_C -= op(X_CR) z with z in the box's z slots (op(X_CR) =
// X_CR, or X_RC^H for the adjoint); backward: t = op(X_RC) x_C into the box's
// t slots (X_RC, or X_CR^H). Rows of C are DOFs idx[r ..], rows of R idx[0 ..].
__device__ __forceinline__ const SolveBox& sv_box(const LevelDev& L, const BoxDesc& d) {
  return L.sbox[&d - L.desc];
}
__device__ __forceinline__ double2 sv_conj(double2 v) { return make_double2(v.x, -v.y); }

template <bool Adj>
struct TcSvC {
  static constexpr bool kConj = false, kUpper = false, kAk = Adj, kBk = true;
  __device__ static bool dims(const LevelDev& L, const BoxDesc& d, const BoxRun&, int& m, int& n,
                              int& k) {
    const SolveBox& B = sv_box(L, d);
    m = B.s + B.n; n = L.snrhs; k = B.r;
    return B.r >= kTcInnerMin && m > 0;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun&, int i, int kk) {
    const SolveBox& B = sv_box(L, d);
    return Adj ? sv_conj(B.XRC[kk + (int64_t)i * B.ldU]) : B.XCR[i + (int64_t)kk * B.ldL];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun&, int kk, int j) {
    return L.spart[j * L.spst + sv_box(L, d).zoff + kk];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun&, const TcExtra&,
                             int i, int j, double vr, double vi) {
    const SolveBox& B = sv_box(L, d);
    double2* p = L.sv + j * L.sn + B.idx[B.r + i];
    const double2 o = *p;
    *p = make_double2(o.x - vr, o.y - vi);
  }
};

template <bool Adj>
struct TcSvT {
  static constexpr bool kConj = false, kUpper = false, kAk = Adj, kBk = true;
  __device__ static bool dims(const LevelDev& L, const BoxDesc& d, const BoxRun&, int& m, int& n,
                              int& k) {
    const SolveBox& B = sv_box(L, d);
    m = B.r; n = L.snrhs; k = B.s + B.n;
    return B.r > 0 && k >= kTcInnerMin;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun&, int i, int kk) {
    const SolveBox& B = sv_box(L, d);
    return Adj ? sv_conj(B.XCR[kk + (int64_t)i * B.ldL]) : B.XRC[i + (int64_t)kk * B.ldU];
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun&, int kk, int j) {
    const SolveBox& B = sv_box(L, d);
    return L.sv[j * L.sn + B.idx[B.r + kk]];
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun&, const TcExtra&,
                             int i, int j, double vr, double vi) {
    L.spart[j * L.spst + sv_box(L, d).toff + i] = make_double2(vr, vi);
  }
};

// an ID-matrix entry as complex128: complex64 entries are widened from their
// bit patterns (integer operations; the conversion instruction would run on
// GB300's narrow fp64 pipe, which it saturated in the split passes)
__device__ __forceinline__ double2 id_entry(double2 v) { return v; }
__device__ __forceinline__ double2 id_entry(float2 v) {
  return make_double2(f2d_bits(v.x), f2d_bits(v.y));
}

// G = M^H M of the ID matrix M (m x a, column-major, ld mmax): a x a x m
template <typename CM>
struct TcGram {
  static constexpr bool kConj = true, kUpper = true, kAk = true, kBk = true;
  __device__ static bool dims(const LevelDev& L, const BoxDesc& d, const BoxRun& rr, int& m,
                              int& n, int& k) {
    m = d.a; n = d.a; k = 2 * rr.nq + 2 * L.n_proxy; return d.a > 0;
  }
  __device__ static double2 A(const LevelDev& L, const BoxDesc& d, const BoxRun&, int i, int kk) {
    return id_entry(reinterpret_cast<const CM*>(L.Mbuf)[d.M_off + kk + (int64_t)i * d.mmax]);
  }
  __device__ static double2 B(const LevelDev& L, const BoxDesc& d, const BoxRun&, int kk, int j) {
    return id_entry(reinterpret_cast<const CM*>(L.Mbuf)[d.M_off + kk + (int64_t)j * d.mmax]);
  }
  __device__ static void epi(const LevelDev& L, const BoxDesc& d, const BoxRun&, const TcExtra& x,
                             int i, int j, double vr, double vi) {
    if (i > j) return;   // the lower triangle is written as the mirror
    const int b = (int)(&d - L.desc);
    double2* G = x.gbuf + x.gb[b].G_off;
    const int a = d.a;
    G[i + (int64_t)j * a] = make_double2(vr, i == j ? 0.0 : vi);
    if (i < j) G[j + (int64_t)i * a] = make_double2(vr, -vi);
  }
};

// The Gram matrix's k range (the rows of M, thousands) is split into chunks
// of 128 k16 steps so that small colours still fill the GPU.
template <typename CM> struct TcSplit<TcGram<CM>> { static constexpr int steps = kGramChunkDefault; };

// G from the split-K int64 accumulator: G_ij = X_hi 2^(E-32) + X_lo 2^(E-16-8 DMAX)
// for i <= j, mirrored to G_ji = conj(G_ij)
template <int DMAX>
__global__ void __launch_bounds__(256) k_gram_finalize(LevelDev L, int b0, const TcUnit* __restrict__ units,
                                                       const TcBoxHost* __restrict__ tb,
                                                       const int* __restrict__ expo, TcExtra x) {
  const TcUnit u = units[blockIdx.y];
  const int b = b0 + u.box;
  const BoxDesc& d = L.desc[b];
  const int64_t a = d.a;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a * a) return;
  const int i = (int)(e % a), j = (int)(e / a);
  if (i > j) return;
  const TcBoxHost t = tb[u.box];
  const unsigned long long* q = x.gx + x.gx_off[b] + 4 * e;
  const int E = expo[t.ea_off + i] + expo[t.eb_off + j];
  const double hr = (double)(long long)q[0], hi = (double)(long long)q[1];
  const double lr = (double)(long long)q[2], li = (double)(long long)q[3];
  const double vr = ldexp(hr, E - 32) + ldexp(lr, E - 16 - 8 * DMAX);
  const double vi = i == j ? 0.0 : ldexp(hi, E - 32) + ldexp(li, E - 16 - 8 * DMAX);
  double2* G = x.gbuf + x.gb[b].G_off;
  G[i + j * a] = make_double2(vr, vi);
  if (i < j) G[j + i * a] = make_double2(vr, -vi);
}

// ---------------------------------------------------------------------------
// split: (1) the power-of-two exponent of every row of A (side 0) / column of
// B (side 1); (2) the digits, each thread converting 8 consecutive k of one
// row into one 16-byte vector per digit and part (32 lanes = 32 consecutive
// rows = 512 contiguous bytes of the core-matrix layout)

template <class Prob>
__device__ __forceinline__ double2 tc_elem(const LevelDev& L, const BoxDesc& d, const BoxRun& rr,
                                           bool side_b, int row, int kk) {
  return side_b ? Prob::B(L, d, rr, kk, row) : Prob::A(L, d, rr, row, kk);
}

// largest component magnitude as the bit pattern of a non-negative double:
// integer max on the magnitude bits orders like the values (NaN above inf)
__device__ __forceinline__ unsigned long long mag_bits(double2 v) {
  const unsigned long long ax = (unsigned long long)__double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long ay = (unsigned long long)__double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFull;
  return ax > ay ? ax : ay;
}

__device__ __forceinline__ int tc_exponent(double mx) {
  int e = 0;
  if (mx > 0.0) {
    frexp(mx, &e);   // mx < 2^e
    e += 1;          // |v| < 2^(e-1): the leading balanced digit stays in [-128, 128]
  }
  return e;
}

template <class Prob, bool SideB>
__device__ __forceinline__ void tc_exp_unit(const LevelDev& L, int b0, const TcBoxHost* __restrict__ tb,
                                            int* expo, const TcUnit& u) {
  const int b = b0 + u.box;
  const BoxDesc& d = L.desc[b];
  const BoxRun rr = L.run[b];
  int m, n, k;
  if (!Prob::dims(L, d, rr, m, n, k)) return;
  const TcBoxHost t = tb[u.box];
  constexpr bool side_b = SideB;
  constexpr bool kcontig = SideB ? Prob::kBk : Prob::kAk;
  const int len = side_b ? n : m;
  const int lpad = side_b ? (n + tc::kCols - 1) / tc::kCols * tc::kCols
                          : (m + tc::kRows - 1) / tc::kRows * tc::kRows;
  int* ex = expo + (side_b ? t.eb_off : t.ea_off);
  const int lane = threadIdx.x & 31;
  if (kcontig) {                 // a warp per row, lanes along k
    const int row = u.x * 8 + (threadIdx.x >> 5);
    if (row >= lpad) return;
    unsigned long long mb = 0;
    if (row < len)
      for (int kk = lane; kk < k; kk += 32) {
        const unsigned long long q = mag_bits(tc_elem<Prob>(L, d, rr, side_b, row, kk));
        mb = q > mb ? q : mb;
      }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long q = __shfl_xor_sync(0xffffffffu, mb, o);
      mb = q > mb ? q : mb;
    }
    double mx = __longlong_as_double((long long)mb);
    if (!(mx <= 1.7976931348623157e308)) {
      if (lane == 0) set_status(L.status, kStatusNonfinite);
      mx = 0.0;
    }
    if (lane == 0) ex[row] = tc_exponent(mx);
  } else {                       // 32 consecutive rows per block, k split over the 8 warps
    __shared__ unsigned long long s_mx[8][32];
    const int warp = threadIdx.x >> 5;
    const int row = u.x * 32 + lane;
    unsigned long long mb = 0;
    if (row < len)
      for (int kk = warp; kk < k; kk += 8) {
        const unsigned long long q = mag_bits(tc_elem<Prob>(L, d, rr, side_b, row, kk));
        mb = q > mb ? q : mb;
      }
    s_mx[warp][lane] = mb;
    __syncthreads();
    if (warp == 0) {
      for (int w = 1; w < 8; ++w) mb = s_mx[w][lane] > mb ? s_mx[w][lane] : mb;
      double mx = __longlong_as_double((long long)mb);
      if (!(mx <= 1.7976931348623157e308)) {
        set_status(L.status, kStatusNonfinite);
        mx = 0.0;
      }
      if (row < lpad) ex[row] = tc_exponent(mx);
    }
  }
}

// one launch for both operands: the unit says which side
template <class Prob>
__global__ void __launch_bounds__(256) k_tc_exp(LevelDev L, int b0, const TcBoxHost* __restrict__ tb,
                                                int* expo, const TcUnit* __restrict__ units) {
  const TcUnit u = units[blockIdx.x];
  if (u.side) tc_exp_unit<Prob, true>(L, b0, tb, expo, u);
  else tc_exp_unit<Prob, false>(L, b0, tb, expo, u);
}

__device__ __forceinline__ uint32_t pack_bf16x2(int lo, int hi) { return tc::bf16_pair(lo, hi); }

template <class Prob> struct TcGramLike { static constexpr bool value = false; };
template <typename CM> struct TcGramLike<TcGram<CM>> { static constexpr bool value = true; };

// grid: x = 32-row groups, y = k-octet groups of 8 (one per warp), z = boxes
template <class Prob, int NS, bool SideB>
__device__ __forceinline__ void tc_digits_unit(const LevelDev& L, int b0,
                                               const TcBoxHost* __restrict__ tb,
                                               unsigned char* slices, const int* __restrict__ expo,
                                               const TcUnit& u) {
  const int b = b0 + u.box;
  const BoxDesc& d = L.desc[b];
  const BoxRun rr = L.run[b];
  int m, n, k;
  if (!Prob::dims(L, d, rr, m, n, k)) return;
  const TcBoxHost t = tb[u.box];
  const int len = SideB ? n : m;
  const int lpad = SideB ? (n + tc::kCols - 1) / tc::kCols * tc::kCols
                         : (m + tc::kRows - 1) / tc::kRows * tc::kRows;
  const int KS = (k + 15) / 16;
  const int row = u.x * 32 + (threadIdx.x & 31);
  const int ko = u.y * 8 + (threadIdx.x >> 5);      // k-octet
  if (ko >= 2 * KS) return;
  if (row >= lpad) return;
  const int e = expo[(SideB ? t.eb_off : t.ea_off) + row];
  int cr[8][NS], ci[8][NS];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int kk = 8 * ko + u;
    double2 v = make_double2(0.0, 0.0);
    if (row < len && kk < k) v = tc_elem<Prob>(L, d, rr, SideB, row, kk);
    if (mag_bits(v) >= 0x7FF0000000000000ull) {   // inf or NaN (exponent bits all set)
      set_status(L.status, kStatusNonfinite);   // NaN escapes the exponent pass's fmax
      v = make_double2(0.0, 0.0);
    }
    tc::balanced_digits<NS>(v.x, e, cr[u]);
    tc::balanced_digits<NS>(v.y, e, ci[u]);
  }
  const int ks = ko >> 1, kc = ko & 1;
  const int ga = tc::a_groups(m), ach = tc::a_chunk(m);
  if (!SideB && (row % tc::kRows) < 8 * ga) {
    const int blk = row / tc::kRows, r = row % tc::kRows;
    unsigned char* step = slices + t.a_off + ((int64_t)blk * KS + ks) * (2 * NS) * ach;
    const int off = (kc * ga + (r >> 3)) * 128 + (r & 7) * 16;
#pragma unroll
    for (int p = 0; p < NS; ++p) {
      uint4 vr, vi;
      vr.x = pack_bf16x2(cr[0][p], cr[1][p]); vr.y = pack_bf16x2(cr[2][p], cr[3][p]);
      vr.z = pack_bf16x2(cr[4][p], cr[5][p]); vr.w = pack_bf16x2(cr[6][p], cr[7][p]);
      vi.x = pack_bf16x2(ci[0][p], ci[1][p]); vi.y = pack_bf16x2(ci[2][p], ci[3][p]);
      vi.z = pack_bf16x2(ci[4][p], ci[5][p]); vi.w = pack_bf16x2(ci[6][p], ci[7][p]);
      *reinterpret_cast<uint4*>(step + (2 * p) * ach + off) = vr;
      *reinterpret_cast<uint4*>(step + (2 * p + 1) * ach + off) = vi;
    }
  }
  // The Gram product's B operand is M itself: column j of B is row j of A
  // (the same exponent and digits), so the A-side unit writes both layouts
  if (SideB || TcGramLike<Prob>::value) {
    const int lpb = (n + tc::kCols - 1) / tc::kCols * tc::kCols;
    if (row >= lpb) return;
    const int blk = row / tc::kCols, r = row % tc::kCols;
    unsigned char* step = slices + t.b_off + ((int64_t)blk * KS + ks) * NS * tc::kBChunk;
    constexpr int rg = 3 * tc::kCols / 8;   // row groups of the three-part block
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      unsigned char* dg = step + q * tc::kBChunk;
      // three 32-row parts: [-im | re | im], or [re | im | -re] for conj(A)
#pragma unroll
      for (int part = 0; part < 3; ++part) {
        int w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int re = cr[u][q], im = ci[u][q];
          w[u] = Prob::kConj ? (part == 0 ? re : part == 1 ? im : -re)
                             : (part == 0 ? -im : part == 1 ? re : im);
        }
        uint4 v;
        v.x = pack_bf16x2(w[0], w[1]); v.y = pack_bf16x2(w[2], w[3]);
        v.z = pack_bf16x2(w[4], w[5]); v.w = pack_bf16x2(w[6], w[7]);
        const int pr = part * tc::kCols + r;
        *reinterpret_cast<uint4*>(dg + (kc * rg + (pr >> 3)) * 128 + (pr & 7) * 16) = v;
      }
    }
  }
}

template <class Prob, int NS>
__global__ void __launch_bounds__(256) k_tc_digits(LevelDev L, int b0, const TcBoxHost* __restrict__ tb,
                                                   unsigned char* slices, const int* __restrict__ expo,
                                                   const TcUnit* __restrict__ units) {
  const TcUnit u = units[blockIdx.x];
  if (u.side) tc_digits_unit<Prob, NS, true>(L, b0, tb, slices, expo, u);
  else tc_digits_unit<Prob, NS, false>(L, b0, tb, slices, expo, u);
}

// ---------------------------------------------------------------------------
// the product: persistent CTAs (one per SM) looping over 128 x 32 complex
// tiles. Barrier phases, window counts and the two-stage operand pipeline
// run on across tiles, so the producer prefetches the next tile while the
// current one drains and the epilogue of one tile overlaps the next tile's
// first MMAs. Every role walks the same unit sequence and skips the same
// units.

struct TcTile {
  bool ok;
  int rel, b, tm, tn, i0, j0, m, n;
  int KSall;   // k16 steps of the whole product
  int k0, KS;  // this unit's chunk of them (split-K problems), else 0 and KSall
};


template <class Prob>
__device__ __forceinline__ TcTile tc_tile(const LevelDev& L, int b0, const TcUnit& u) {
  TcTile T;
  T.ok = false;
  T.rel = u.box;
  T.b = b0 + u.box;
  int m, n, k;
  if (!Prob::dims(L, L.desc[T.b], L.run[T.b], m, n, k)) return T;
  const int tms = (m + tc::kRows - 1) / tc::kRows, tns = (n + tc::kCols - 1) / tc::kCols;
  if (u.x >= tms * tns) return T;
  T.tm = u.x % tms;
  T.tn = u.x / tms;
  T.i0 = T.tm * tc::kRows;
  T.j0 = T.tn * tc::kCols;
  if (Prob::kUpper && T.j0 + tc::kCols - 1 < T.i0) return T;   // below the diagonal
  T.m = m;
  T.n = n;
  T.KSall = (k + 15) / 16;
  T.k0 = 0;
  T.KS = T.KSall;
  if (TcSplit<Prob>::steps > 0) {
    // chunk length: from the unit (product units of a split-K problem carry
    // it in `side`), else the problem's default
    const int cs = u.side > 0 ? u.side : TcSplit<Prob>::steps;
    T.k0 = u.y * cs;
    if (T.k0 >= T.KSall) return T;   // past the end of this box's k range
    T.KS = min(cs, T.KSall - T.k0);
  }
  T.ok = true;
  return T;
}

template <class Prob, int NS, int DMAX>
__global__ void __launch_bounds__(tc::kThreads, 1)
    k_tc_gemm(LevelDev L, int b0, const TcBoxHost* __restrict__ tb,
              const unsigned char* __restrict__ slices, const int* __restrict__ expo, TcExtra x,
              const TcUnit* __restrict__ units, int nunits) {
  using namespace tc;
  constexpr int kA = NS * 2 * kAChunk, kB = NS * kBChunk, kStage = kA + kB;
  constexpr int kAcc = DMAX + 1;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[2], bar_empty[2], bar_accf[kAcc], bar_accr[kAcc], bar_done;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  unsigned char* sm =
      reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) { mbar_init(&bar_full[s], 1); mbar_init(&bar_empty[s], 1); }
    for (int a = 0; a < kAcc; ++a) { mbar_init(&bar_accf[a], 1); mbar_init(&bar_accr[a], 8); }
    mbar_init(&bar_done, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&s_tmem)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  volatile int* abort_flag = &s_abort;

  if (warp == 0) {
    // ---- producer: two-stage bulk-copy pipeline over all steps of all tiles
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int ui = blockIdx.x; ui < nunits && ok; ui += gridDim.x) {
        const TcTile T = tc_tile<Prob>(L, b0, units[ui]);
        if (!T.ok) continue;
        const TcBoxHost t = tb[T.rel];
        const int kAt = NS * 2 * a_chunk(T.m);   // this tile's A bytes per k16 step
        const unsigned char* srcA = slices + t.a_off + ((int64_t)T.tm * T.KSall + T.k0) * kAt;
        const unsigned char* srcB = slices + t.b_off + ((int64_t)T.tn * T.KSall + T.k0) * kB;
        for (int ks = 0; ks < T.KS; ++ks, ++g) {
          const int s = g & 1;
          if (g >= 2 && !mbar_wait(&bar_empty[s], ((g >> 1) - 1) & 1, abort_flag)) { ok = false; break; }
          unsigned char* st = sm + s * kStage;
          mbar_expect_tx(&bar_full[s], (uint32_t)(kAt + kB));
          bulk_g2s(st, srcA + (int64_t)ks * kAt, (uint32_t)kAt, &bar_full[s]);
          bulk_g2s(st + kA, srcB + (int64_t)ks * kB, (uint32_t)kB, &bar_full[s]);
        }
      }
      if (*abort_flag) {
        // let the copies in flight land before the CTA's shared memory goes away
        for (int gg = g > 2 ? g - 2 : 0; gg < g; ++gg)
          for (long long i = 0; i < kWaitLimit; ++i)
            if (mbar_try(&bar_full[gg & 1], (gg >> 1) & 1)) break;
      }
    }
  } else if (warp == 1) {
    // ---- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t smem0 = su32(sm);
      const uint32_t boffA = Prob::kConj ? 0u : 512u;   // B rows for the A_re product
      const uint32_t boffB = Prob::kConj ? 512u : 0u;   // B rows for the A_im product
      const uint64_t dB = sdesc(0, 1536, 128);
      // per accumulator: bit d of `opened` = a window of d was opened before,
      // bit d of `wpar` = parity of the number of windows of d opened
      uint32_t opened = 0, wpar = 0;
      int g = 0;
      bool ok = true;
      for (int ui = blockIdx.x; ui < nunits && ok; ui += gridDim.x) {
        const TcTile T = tc_tile<Prob>(L, b0, units[ui]);
        if (!T.ok) continue;
        const int ach = a_chunk(T.m);
        const uint64_t dA = sdesc(0, (uint32_t)(a_groups(T.m) * 128), 128);
        for (int ks = 0; ks < T.KS && ok; ++ks, ++g) {
          const int s = g & 1;
          if (!mbar_wait(&bar_full[s], (g >> 1) & 1, abort_flag)) { ok = false; break; }
          fence_after();
          const uint32_t aS = smem0 + s * kStage, bS = aS + kA;
#pragma unroll
          for (int dd = 0; dd < kAcc; ++dd) {
            const int W = window(dd, NS);
            const bool start = ks % W == 0;
            if (start && ((opened >> dd) & 1u)) {
              // the drain of the previous window: phase (windows opened - 1)
              if (!mbar_wait(&bar_accr[dd], ((wpar >> dd) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
              fence_after();
            }
            if (start) { opened |= 1u << dd; wpar ^= 1u << dd; }
            const uint32_t dt = tmem + 64 * dd;
            uint32_t acc = start ? 0u : 1u;
            for (int p = plo(dd, NS); p <= phi(dd, NS); ++p) {
              const int q = dd - p;
              const uint32_t ar = aS + (2 * p) * ach, ai = ar + ach;
              const uint32_t bq = bS + q * kBChunk;
              mma(dt, dA + (ar >> 4), dB + ((bq + boffA) >> 4), acc);
              mma(dt, dA + (ai >> 4), dB + ((bq + boffB) >> 4), 1u);
              acc = 1u;
            }
            if ((ks + 1) % W == 0 || ks == T.KS - 1) commit(&bar_accf[dd]);
          }
          if (!ok) break;
          commit(&bar_empty[s]);
        }
      }
      // all MMAs issued by this thread complete before tensor memory is freed
      commit(&bar_done);
      for (long long i = 0; i < kWaitLimit; ++i)
        if (mbar_try(&bar_done, 0)) break;
    }
  } else {
    // ---- epilogue: drain each accumulator window into 64-bit integers
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int half = ew >> 2;
    const int row = 32 * quarter + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16);
    uint32_t dpar = 0;   // bit d: parity of the number of windows of d drained
    bool ok = true;
    for (int ui = blockIdx.x; ui < nunits && ok; ui += gridDim.x) {
      const TcTile T = tc_tile<Prob>(L, b0, units[ui]);
      if (!T.ok) continue;
      long long xh[16][2], xl[16][2];
#pragma unroll
      for (int c = 0; c < 16; ++c) xh[c][0] = xh[c][1] = xl[c][0] = xl[c][1] = 0;
      for (int ks = 0; ks < T.KS && ok; ++ks) {
#pragma unroll
        for (int dd = 0; dd < kAcc; ++dd) {
          const int W = window(dd, NS);
          if (!((ks + 1) % W == 0 || ks == T.KS - 1)) continue;
          if (!mbar_wait(&bar_accf[dd], (dpar >> dd) & 1u, abort_flag)) { ok = false; break; }
          dpar ^= 1u << dd;
          fence_after();
          float vr[16], vi[16];
          tmem_ld16(tl + 64 * dd + 16 * half, vr);
          tmem_ld16(tl + 64 * dd + 32 + 16 * half, vi);
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bar_accr[dd]);
          const bool hi = dd <= 2;
          const int sh = hi ? 8 * (2 - dd) : 8 * (DMAX - dd);
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const long long r0 = (long long)__float2int_rn(vr[c]) << sh;
            const long long r1 = (long long)__float2int_rn(vi[c]) << sh;
            if (hi) { xh[c][0] += r0; xh[c][1] += r1; }
            else { xl[c][0] += r0; xl[c][1] += r1; }
          }
        }
      }
      if (!ok || *abort_flag) break;
      const int i = T.i0 + row;
      if (TcSplit<Prob>::steps > 0) {
        // add this chunk's exact digit sums into the box's int64 accumulator
        if (i < T.m) {
          const BoxDesc& d = L.desc[T.b];
          unsigned long long* acc = x.gx + x.gx_off[T.b];
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int j = T.j0 + 16 * half + c;
            if (j >= T.n || (Prob::kUpper && i > j)) continue;
            unsigned long long* q = acc + 4 * ((int64_t)i + (int64_t)j * d.a);
            atomicAdd(q + 0, (unsigned long long)xh[c][0]);
            atomicAdd(q + 1, (unsigned long long)xh[c][1]);
            atomicAdd(q + 2, (unsigned long long)xl[c][0]);
            atomicAdd(q + 3, (unsigned long long)xl[c][1]);
          }
        }
        continue;
      }
      if (i < T.m) {
        const TcBoxHost t = tb[T.rel];
        const BoxDesc& d = L.desc[T.b];
        const BoxRun rr = L.run[T.b];
        const int ei = expo[t.ea_off + i];
        [[maybe_unused]] typename std::conditional<TcRowEpi<Prob>::value, Prob, TcNoRow>::type::Row
            w;
        if constexpr (TcRowEpi<Prob>::value) w = Prob::row(L, d, rr, i);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int j = T.j0 + 16 * half + c;
          if (j >= T.n) continue;
          const int E = ei + expo[t.eb_off + j];
          // value = X_hi 2^(E - 32) + X_lo 2^(E - 16 - 8 DMAX); the powers of two
          // are built from their bits (GB300's fp64 pipe is the scarce unit)
          const int bh = E - 32 + 1023, bl = E - 16 - 8 * DMAX + 1023;
          double vr, vi;
          if (bl >= 1 && bh <= 2046) {
            const double sh = __longlong_as_double((long long)bh << 52);
            const double sl = __longlong_as_double((long long)bl << 52);
            vr = fma((double)xl[c][0], sl, (double)xh[c][0] * sh);
            vi = fma((double)xl[c][1], sl, (double)xh[c][1] * sh);
          } else {
            vr = ldexp((double)xh[c][0], E - 32) + ldexp((double)xl[c][0], E - 16 - 8 * DMAX);
            vi = ldexp((double)xh[c][1], E - 32) + ldexp((double)xl[c][1], E - 16 - 8 * DMAX);
          }
          if constexpr (TcRowEpi<Prob>::value) Prob::col(L, w, j, vr, vi);
          else Prob::epi(L, d, rr, x, i, j, vr, vi);
        }
      }
    }
  }
  __syncthreads();
  if (*abort_flag && tid == 0) set_status(L.status, kStatusTimeout);
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
}

// ---------------------------------------------------------------------------
// host side

size_t tc_smem_bytes(int ns) {
  // at least 120 KB so that one CTA (holding all 512 tensor-memory columns)
  // runs per SM
  return std::max<size_t>((size_t)2 * (ns * 2 * tc::kAChunk + ns * tc::kBChunk) + 1024,
                          (size_t)120 * 1024);
}

void plan_tc_box(int mrows, int ncols, int k, int ns, int64_t& slice_off, int64_t& expo_off,
                 TcBoxHost& out) {
  const int64_t ks = (k + 15) / 16;
  const int64_t mb = (mrows + tc::kRows - 1) / tc::kRows, nb = (ncols + tc::kCols - 1) / tc::kCols;
  out.a_off = slice_off;
  slice_off += mb * ks * ns * 2 * tc::kAChunk;
  out.b_off = slice_off;
  slice_off += nb * ks * ns * tc::kBChunk;
  out.ea_off = expo_off;
  expo_off += mb * tc::kRows;
  out.eb_off = expo_off;
  expo_off += nb * tc::kCols;
}

// Sizes of problem `which` for one box: the same rules as the device-side
// dims() of the problem structs (which the kernels re-check).
static bool tc_dims_host(int which, const TcBoxSize& z, int& m, int& n, int& k) {
  switch (which) {
    case kTcG1: m = z.r; n = z.a + z.n; k = z.s; return z.r > 0 && z.s >= kTcInnerMin;
    case kTcG3: m = z.a + z.n; n = z.r; k = z.s; return z.r > 0 && z.s >= kTcInnerMin;
    case kTcW: m = z.s + z.n; n = z.r; k = z.r; return z.r >= kTcInnerMin;
    case kTcSchur: m = z.s + z.n; n = m; k = z.r; return z.r >= kTcInnerMin;
    case kTcXrr: m = z.r; n = z.r; k = z.s; return z.r > 0 && z.s >= kTcInnerMin;
    case kTcGram: m = z.a; n = z.a; k = z.kgram; return z.a > 0;
    case kTcNsY:
    case kTcNsX: m = z.r; n = z.r; k = z.r; return z.r >= kNsMin && z.r <= z.nsmax;
    // root step: a = later DOFs, r = block width
    case kTcRootW: m = z.a; n = z.r; k = z.r; return z.a > 0 && z.r >= kTcInnerMin;
    case kTcRootS: m = z.a; n = z.a; k = z.r; return z.a > 0 && z.r >= kTcInnerMin;
    // solve sweeps (per colour of the solve plan)
    case kTcSvC:
    case kTcSvCA: m = z.s + z.n; n = z.nrhs; k = z.r; return z.r >= kTcInnerMin && m > 0;
    case kTcSvT:
    case kTcSvTA: m = z.r; n = z.nrhs; k = z.s + z.n; return z.r > 0 && k >= kTcInnerMin;
  }
  return false;
}

static bool tc_kcontig(int which, bool side_b) {
  return side_b || which == kTcG1 || which == kTcGram || which == kTcSvCA || which == kTcSvTA;
}

void tc_plan(int which, const std::vector<TcBoxSize>& boxes, std::vector<TcUnit>& units,
             TcPlan& plan, int gram_chunk) {
  if (gram_chunk < 1) gram_chunk = kGramChunkDefault;
  for (int l = 0; l < 5; ++l) {
    plan.off[l] = (int)units.size();
    for (int e = 0; e < (int)boxes.size(); ++e) {
      int m, n, k;
      if (!tc_dims_host(which, boxes[e], m, n, k)) continue;
      const int lpa = (m + tc::kRows - 1) / tc::kRows * tc::kRows;
      const int lpb = (n + tc::kCols - 1) / tc::kCols * tc::kCols;
      const int kg = (2 * ((k + 15) / 16) + 7) / 8;
      if (l < 2) {                       // exponents of side A / B
        // (the Gram product's B exponents are its A exponents: not recomputed)
        if (l == 1 && which == kTcGram) continue;
        const int lp = l == 0 ? lpa : lpb;
        const int per = tc_kcontig(which, l == 1) ? 8 : 32;
        for (int x = 0; x < (lp + per - 1) / per; ++x) units.push_back(TcUnit{e, l, x, 0});
      } else if (l < 4) {                // digits of side A / B
        // (the Gram product's A-side units write the B digits too)
        if (l == 3 && which == kTcGram) continue;
        const int lp = l == 2 ? lpa : lpb;
        for (int x = 0; x < lp / 32; ++x)
          for (int y = 0; y < kg; ++y) units.push_back(TcUnit{e, l - 2, x, y});
      } else {                           // product tiles (and k chunks of the Gram matrix)
        const int tms = lpa / tc::kRows, tns = lpb / tc::kCols;
        const int nchunk = which == kTcGram ? ((k + 15) / 16 + gram_chunk - 1) / gram_chunk : 1;
        const int cs = which == kTcGram ? gram_chunk : 0;
        for (int t = 0; t < tms * tns; ++t) {
          const int i0 = (t % tms) * tc::kRows, j0 = (t / tms) * tc::kCols;
          if (which == kTcGram && j0 + tc::kCols - 1 < i0) continue;
          for (int c = 0; c < nchunk; ++c) units.push_back(TcUnit{e, cs, t, c});
        }
      }
    }
    plan.cnt[l] = (int)units.size() - plan.off[l];
  }
}

template <class Prob, int NS, int DMAX>
static void launch_tc(const char* name, const LevelDev& L, int b0, const TcBoxHost* d_tb,
                      void* slices, int* expo, const TcExtra& x, const TcUnit* d_units,
                      const TcPlan& pl, cudaStream_t st) {
  unsigned char* sl = reinterpret_cast<unsigned char*>(slices);
  // the exponent units of both sides are adjacent in the list, so are the digit units
  const int ne = pl.cnt[0] + pl.cnt[1], nd = pl.cnt[2] + pl.cnt[3];
  if (ne > 0)
    FMMLU_LAUNCH("tc_split", st,
                 (k_tc_exp<Prob><<<ne, 256, 0, st>>>(L, b0, d_tb, expo, d_units + pl.off[0])));
  if (nd > 0)
    FMMLU_LAUNCH("tc_split", st,
                 (k_tc_digits<Prob, NS><<<nd, 256, 0, st>>>(L, b0, d_tb, sl, expo, d_units + pl.off[2])));
  if (pl.cnt[4] <= 0) return;
  const size_t smem = tc_smem_bytes(NS);
  // the shared-memory limit is a per-device attribute: set it once per device
  int dev = 0;
  cudaGetDevice(&dev);
  static std::once_flag attr_once[64];
  if (dev >= 0 && dev < 64)
    std::call_once(attr_once[dev], [smem] {
      cudaFuncSetAttribute(k_tc_gemm<Prob, NS, DMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    });
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(pl.cnt[4], std::max(sms, 1));   // one persistent CTA per SM
  FMMLU_LAUNCH(name, st,
               (k_tc_gemm<Prob, NS, DMAX><<<grid, tc::kThreads, smem, st>>>(
                   L, b0, d_tb, sl, expo, x, d_units + pl.off[4], pl.cnt[4])));
}

void launch_tc_planned(int which, const LevelDev& L, int b0, const TcBoxHost* d_tb, void* slices,
                       int* expo, const GramBoxHost* d_gb, double2* gbuf, bool fp32,
                       const TcUnit* d_units, const TcPlan& pl, cudaStream_t st,
                       unsigned long long* gx, const int64_t* gx_off) {
  const TcExtra x{d_gb, gbuf, gx, gx_off};
  switch (which) {
    case kTcG1: launch_tc<TcG1, 7, 6>("gemm_g1_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcG3: launch_tc<TcG3, 7, 6>("gemm_g3_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcW: launch_tc<TcW, 7, 6>("gemm_w_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcSchur: launch_tc<TcSchur, 7, 6>("schur_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcXrr: launch_tc<TcXrr, 7, 6>("gemm_xrr_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcNsY: launch_tc<TcNsY, 7, 6>("ns_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcNsX: launch_tc<TcNsX, 7, 6>("ns_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcRootW: launch_tc<TcRootW, 7, 6>("root_w_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcRootS: launch_tc<TcRootS, 7, 6>("root_schur_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcSvC: launch_tc<TcSvC<false>, 7, 6>("sweep_c_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcSvCA: launch_tc<TcSvC<true>, 7, 6>("sweep_c_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcSvT: launch_tc<TcSvT<false>, 7, 6>("sweep_t_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcSvTA: launch_tc<TcSvT<true>, 7, 6>("sweep_t_tc", L, b0, d_tb, slices, expo, x, d_units, pl, st); break;
    case kTcGram:
      if (fp32) launch_tc<TcGram<float2>, 4, 4>("gram", L, b0, d_tb, slices, expo, x, d_units, pl, st);
      else launch_tc<TcGram<double2>, 7, 6>("gram", L, b0, d_tb, slices, expo, x, d_units, pl, st);
      break;
  }
}

void launch_gram_finalize(const LevelDev& L, int b0, const TcUnit* d_boxes, int nboxes, int amax,
                          const TcBoxHost* d_tb, const int* expo, const GramBoxHost* d_gb,
                          double2* gbuf, unsigned long long* gx, const int64_t* gx_off, bool fp32,
                          cudaStream_t st) {
  if (nboxes <= 0) return;
  const TcExtra x{d_gb, gbuf, gx, gx_off};
  dim3 grid((unsigned)(((int64_t)amax * amax + 255) / 256), (unsigned)nboxes);
  if (fp32)
    FMMLU_LAUNCH("gram", st, (k_gram_finalize<4><<<grid, 256, 0, st>>>(L, b0, d_boxes, d_tb, expo, x)));
  else
    FMMLU_LAUNCH("gram", st, (k_gram_finalize<6><<<grid, 256, 0, st>>>(L, b0, d_boxes, d_tb, expo, x)));
}

// ---------------------------------------------------------------------------
// the root factor with its two products per step on the tensor cores: the
// diagonal-block inverses stay fp64 Gauss-Jordan (launch_root_diag); all
// steps' unit lists are known up front and uploaded once.

cudaError_t launch_root_factor_tc(double2* A, int n0, int nb, double2* W, int* status,
                                  cudaStream_t st) {
  struct Step { int i0, r; TcPlan pw, ps; };
  std::vector<Step> steps;
  std::vector<TcUnit> units;
  for (int i0 = 0; i0 < n0; i0 += nb) {
    Step sp;
    sp.i0 = i0;
    sp.r = std::min(nb, n0 - i0);
    const std::vector<TcBoxSize> bs{TcBoxSize{n0 - i0 - sp.r, 0, sp.r, 0, 0, 0}};
    tc_plan(kTcRootW, bs, units, sp.pw);
    tc_plan(kTcRootS, bs, units, sp.ps);
    steps.push_back(sp);
  }
  int64_t so = 0, eo = 0;
  TcBoxHost tb;
  plan_tc_box(n0, n0, nb, 7, so, eo, tb);
  void *d_slices = nullptr, *d_expo = nullptr, *d_units = nullptr, *d_tb = nullptr,
       *d_desc = nullptr, *d_run = nullptr;
  auto cleanup = [&]() {
    for (void* p : {d_slices, d_expo, d_units, d_tb, d_desc, d_run}) if (p) cudaFree(p);
  };
  cudaError_t err = cudaSuccess;
  auto ck = [&](cudaError_t e) {
    if (err == cudaSuccess && e != cudaSuccess) err = e;
    return err == cudaSuccess;
  };
  if (!(ck(cudaMalloc(&d_slices, (size_t)std::max<int64_t>(so, 16))) &&
        ck(cudaMalloc(&d_expo, (size_t)std::max<int64_t>(eo, 1) * sizeof(int))) &&
        ck(cudaMalloc(&d_units, std::max<size_t>(units.size(), 1) * sizeof(TcUnit))) &&
        ck(cudaMalloc(&d_tb, sizeof(TcBoxHost))) && ck(cudaMalloc(&d_desc, sizeof(BoxDesc))) &&
        ck(cudaMalloc(&d_run, sizeof(BoxRun))) &&
        ck(cudaMemsetAsync(d_desc, 0, sizeof(BoxDesc), st)) &&
        ck(cudaMemsetAsync(d_run, 0, sizeof(BoxRun), st)) &&
        ck(cudaMemcpyAsync(d_tb, &tb, sizeof(TcBoxHost), cudaMemcpyHostToDevice, st)) &&
        (units.empty() || ck(cudaMemcpyAsync(d_units, units.data(), units.size() * sizeof(TcUnit),
                                             cudaMemcpyHostToDevice, st))))) {
    cudaStreamSynchronize(st);
    cleanup();
    return err;
  }
  LevelDev L{};
  L.desc = reinterpret_cast<const BoxDesc*>(d_desc);
  L.run = reinterpret_cast<BoxRun*>(d_run);
  L.status = status;
  L.root_A = A;
  L.root_W = W;
  L.root_n0 = n0;
  const TcUnit* du = reinterpret_cast<const TcUnit*>(d_units);
  for (const Step& sp : steps) {
    launch_root_diag(A, n0, sp.i0, sp.r, status, st);
    if (n0 - sp.i0 - sp.r <= 0) continue;
    L.root_i0 = sp.i0;
    L.root_r = sp.r;
    launch_tc_planned(kTcRootW, L, 0, reinterpret_cast<const TcBoxHost*>(d_tb), d_slices,
                      reinterpret_cast<int*>(d_expo), nullptr, nullptr, false, du, sp.pw, st,
                      nullptr, nullptr);
    launch_tc_planned(kTcRootS, L, 0, reinterpret_cast<const TcBoxHost*>(d_tb), d_slices,
                      reinterpret_cast<int*>(d_expo), nullptr, nullptr, false, du, sp.ps, st,
                      nullptr, nullptr);
  }
  ck(cudaGetLastError());
  ck(cudaStreamSynchronize(st));   // the buffers above are freed next
  cleanup();
  return err;
}

}  // namespace fmmlu
