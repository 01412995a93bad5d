// Octree construction (Sec. 4 preamble, Sec. 4.3), all on the GPU.
//
// 1. Bounding cube (min/max reduction; the host forms centre and side from the
//    exact extrema), integer coordinates q = floor((x - corner)/side * 2^21)
//    (clipped to [0, 2^21 - 1]), 63-bit Morton keys (bit 3b <- x_b, 3b+1 <- y_b,
//    3b+2 <- z_b) and a stable LSD radix sort of (key, index) pairs, so equal
//    keys keep the input order.
// 2. Hierarchy, level by level: a box holding more than s points (below the
//    depth cap 21) gets one child per non-empty octant; the octant ranges of
//    its sorted point range are found by binary search on the key digits.
//    Every box is entered in a hash table keyed by its location code
//    (1 << 3l | Morton prefix of its cell).
// 3. Level restriction of Sec. 4 -- a leaf touching (face, edge or corner) a
//    leaf two or more levels finer is split -- in rounds until nothing
//    changes: every leaf F looks at the 26 cells around it at its own level,
//    finds the leaf containing each (the first box that exists walking up the
//    levels) and marks it when it is two or more levels coarser (and below
//    level 20); the marked leaves are split. The result is the minimal
//    balanced refinement, the same whatever the order of splits.
// 4. Box ids ordered by (level, Morton) = (level, first point) by a radix
//    sort; parents and children renumbered.
// 5. For every level l >= 2 (current boxes: the level-l boxes plus all coarser
//    leaves): one thread per level box visits the 5 x 5 x 5 cells around it,
//    finds the current box containing each, and sorts the distinct ones by
//    first point: N(B) = those touching B, Q(B) = those at max-norm gap in
//    (0, h_l]. Two passes (counts, then lists at scanned offsets).
// 6. Colours, greedy in Morton order over the conflict relation gap <= h_l or
//    a shared coarser leaf in the near lists: every box's earlier
//    conflicting boxes are listed in parallel, then one warp per level walks
//    the level's boxes in order and gives each the smallest colour none of
//    its listed boxes has.
// The host downloads the finished arrays into its description of the tree.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>

#include "fmmlu_internal.h"
#include "tree_host.h"

namespace fmmlu {

// ---------------------------------------------------------------------------
// GPU: Morton keys and radix sort
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t spread3(uint64_t v) {
  // spread the low 21 bits of v so that bit b lands at bit 3b
  v &= 0x1fffffULL;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}

__global__ void k_morton(const double* __restrict__ pts, int64_t n, double c0,
                         double c1, double c2, double side, uint64_t* keys,
                         int* idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double one = 2097152.0;  // 2^21
  double c[3] = {c0, c1, c2};
  uint64_t q[3];
  for (int a = 0; a < 3; ++a) {
    // explicit round-to-nearest ops: no contraction, same as the reference
    double t = __dmul_rn(__ddiv_rn(__dsub_rn(pts[3 * i + a], c[a]), side), one);
    double f = floor(t);
    if (!(f >= 0.0)) f = 0.0;
    if (f > one - 1.0) f = one - 1.0;
    q[a] = (uint64_t)f;
  }
  keys[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
  idx[i] = (int)i;
}

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                             int* hist, int nblk) {
  __shared__ int cnt[16];
  if (threadIdx.x < 16) cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kSortTile + threadIdx.x * kSortItems;
  for (int e = 0; e < kSortItems; ++e) {
    int64_t i = base + e;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 15], 1);
  }
  __syncthreads();
  if (threadIdx.x < 16) hist[threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive scan of a small int array in one block (len <= 1M)
__global__ void k_scan_small(int* a, int len) {
  __shared__ int part[1024];
  int t = threadIdx.x;
  int per = (len + blockDim.x - 1) / blockDim.x;
  int b = t * per, e = min(len, b + per);
  int s = 0;
  for (int i = b; i < e; ++i) s += a[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) { int v = part[i]; part[i] = run; run += v; }
  }
  __syncthreads();
  int run = part[t];
  for (int i = b; i < e; ++i) { int v = a[i]; a[i] = run; run += v; }
}

__global__ void k_radix_scatter(const uint64_t* __restrict__ kin, const int* __restrict__ vin,
                                int64_t n, int shift, const int* __restrict__ offs,
                                int nblk, uint64_t* kout, int* vout) {
  __shared__ int cnt[16][kSortThreads];
  __shared__ int warp_tot[16][kSortThreads / 32];
  int t = threadIdx.x;
  int64_t base = (int64_t)blockIdx.x * kSortTile + t * kSortItems;
  int my[16];
  for (int d = 0; d < 16; ++d) my[d] = 0;
  for (int e = 0; e < kSortItems; ++e) {
    int64_t i = base + e;
    if (i < n) my[(kin[i] >> shift) & 15]++;
  }
  // exclusive scan over threads for each digit
  int lane = t & 31, wid = t >> 5;
  for (int d = 0; d < 16; ++d) {
    int v = my[d];
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    cnt[d][t] = incl - v;
    if (lane == 31) warp_tot[d][wid] = incl;
  }
  __syncthreads();
  if (t < 16) {
    int run = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) { int v = warp_tot[t][w]; warp_tot[t][w] = run; run += v; }
  }
  __syncthreads();
  int pos[16];
  for (int d = 0; d < 16; ++d) pos[d] = offs[d * nblk + blockIdx.x] + warp_tot[d][wid] + cnt[d][t];
  for (int e = 0; e < kSortItems; ++e) {
    int64_t i = base + e;
    if (i < n) {
      uint64_t k = kin[i];
      int d = (k >> shift) & 15;
      int p = pos[d]++;
      kout[p] = k;
      vout[p] = vin[i];
    }
  }
}


// ---------------------------------------------------------------------------
// bounding box: per-block extrema of each axis, then one block combines them
// ---------------------------------------------------------------------------

constexpr int kBoxThreads = 256;

__global__ void k_extrema(const double* __restrict__ pts, int64_t n, double* part, int* bad) {
  __shared__ double s[6][kBoxThreads];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int a = 0; a < 3; ++a) {
      const double v = pts[3 * i + a];
      if (!isfinite(v)) *bad = 1;
      lo[a] = fmin(lo[a], v);
      hi[a] = fmax(hi[a], v);
    }
  for (int a = 0; a < 3; ++a) { s[a][threadIdx.x] = lo[a]; s[3 + a][threadIdx.x] = hi[a]; }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int a = 0; a < 3; ++a) {
        s[a][threadIdx.x] = fmin(s[a][threadIdx.x], s[a][threadIdx.x + w]);
        s[3 + a][threadIdx.x] = fmax(s[3 + a][threadIdx.x], s[3 + a][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k_extrema_final(double* part, int nblk) {
  if (threadIdx.x != 0) return;
  for (int b = 1; b < nblk; ++b)
    for (int a = 0; a < 3; ++a) {
      part[a] = fmin(part[a], part[6 * b + a]);
      part[3 + a] = fmax(part[3 + a], part[6 * b + 3 + a]);
    }
}

// ---------------------------------------------------------------------------
// location codes and the box hash table
// ---------------------------------------------------------------------------

// inverse of spread3: bits 0, 3, 6, ... of v packed into the low 21 bits
__host__ __device__ __forceinline__ uint64_t compact3(uint64_t v) {
  v &= 0x1249249249249249ULL;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ULL;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00fULL;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffULL;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffULL;
  v = (v ^ (v >> 32)) & 0x1fffffULL;
  return v;
}

// location code of the level-l cell (x, y, z): a leading 1 above the 3l bits
// of its Morton index, unique over all levels (never 0)
__device__ __forceinline__ uint64_t loc_code(int l, uint64_t x, uint64_t y, uint64_t z) {
  return (1ull << (3 * l)) | spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

__device__ __forceinline__ void cell_of(uint64_t code, int l, int64_t& x, int64_t& y, int64_t& z) {
  const uint64_t m = code & ((1ull << (3 * l)) - 1);   // l <= 21: the shift stays below 64
  x = (int64_t)compact3(m);
  y = (int64_t)compact3(m >> 1);
  z = (int64_t)compact3(m >> 2);
}

struct DHash {
  unsigned long long* keys;   // 0 = empty slot
  int* vals;
  uint32_t mask;              // capacity - 1 (a power of two)
};

__device__ __forceinline__ uint32_t hash_slot(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdULL;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ULL;
  k ^= k >> 33;
  return (uint32_t)k;
}

// false when the table is full (the caller reports it)
__device__ __forceinline__ bool hash_insert(DHash h, uint64_t key, int val) {
  uint32_t s = hash_slot(key) & h.mask;
  for (uint32_t probe = 0; probe <= h.mask; ++probe) {
    const unsigned long long prev = atomicCAS(&h.keys[s], 0ull, (unsigned long long)key);
    if (prev == 0ull || prev == key) {
      h.vals[s] = val;
      return true;
    }
    s = (s + 1) & h.mask;
  }
  return false;
}

__device__ __forceinline__ int hash_find(DHash h, uint64_t key) {
  uint32_t s = hash_slot(key) & h.mask;
  for (uint32_t probe = 0; probe <= h.mask; ++probe) {
    const unsigned long long k = h.keys[s];
    if (k == key) return h.vals[s];
    if (k == 0ull) return -1;
    s = (s + 1) & h.mask;
  }
  return -1;
}

// box arrays (structure of arrays, capacity `cap`)
struct DBoxes {
  int* lvl;
  unsigned long long* code;
  int* start;
  int* end;
  int* parent;
  int* nkids;
  int* mark;
  int* first_kid;
};

// non-empty octants of box i at the next level: child c covers keys
// [cs[c], cs[c + 1]) of the box's sorted range (the octant digits of the
// range are non-decreasing); returns the number of children
__device__ __forceinline__ int octant_ranges(const uint64_t* __restrict__ keys, int s, int e,
                                             int l, int* cs, int* oc) {
  const int shift = 3 * (20 - l);   // digit of level l + 1
  int cnt = 0;
  int lo = s;
  for (int o = 0; o < 8 && lo < e; ++o) {
    // first index in [lo, e) whose digit exceeds o
    int a = lo, b = e;
    while (a < b) {
      const int mid = (a + b) >> 1;
      if ((int)((keys[mid] >> shift) & 7) <= o) a = mid + 1; else b = mid;
    }
    if (a > lo) {
      cs[cnt] = lo;
      oc[cnt] = o;
      ++cnt;
    }
    lo = a;
  }
  cs[cnt] = e;
  return cnt;
}

__device__ __forceinline__ bool splits(const DBoxes& B, int i, int leaf_size) {
  const int l = B.lvl[i];
  return B.end[i] - B.start[i] > leaf_size && l < 21;
}

// hierarchy, level l: children counts of the boxes [b0, b1)
__global__ void k_child_count(DBoxes B, const uint64_t* __restrict__ keys, int b0, int b1,
                              int leaf_size, int* cnt) {
  const int i = b0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b1) return;
  int c = 0;
  if (splits(B, i, leaf_size)) {
    int cs[9], oc[8];
    c = octant_ranges(keys, B.start[i], B.end[i], B.lvl[i], cs, oc);
  }
  cnt[i - b0] = c;
}

__device__ __forceinline__ bool write_children(DBoxes B, DHash H, const uint64_t* keys, int i,
                                               int base) {
  int cs[9], oc[8];
  const int l = B.lvl[i];
  const int c = octant_ranges(keys, B.start[i], B.end[i], l, cs, oc);
  bool ok = true;
  for (int j = 0; j < c; ++j) {
    const int t = base + j;
    B.lvl[t] = l + 1;
    B.code[t] = (B.code[i] << 3) | (unsigned long long)oc[j];
    B.start[t] = cs[j];
    B.end[t] = cs[j + 1];
    B.parent[t] = i;
    B.nkids[t] = 0;
    B.mark[t] = 0;
    ok = hash_insert(H, B.code[t], t) && ok;
  }
  B.nkids[i] = c;
  return ok;
}

// hierarchy, level l: the children of the boxes [b0, b1) at base + off[i - b0]
__global__ void k_child_write(DBoxes B, DHash H, const uint64_t* __restrict__ keys, int b0,
                              int b1, int leaf_size, const int* __restrict__ off, int base,
                              int* fail) {
  const int i = b0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b1 || !splits(B, i, leaf_size)) return;
  if (!write_children(B, H, keys, i, base + off[i - b0])) *fail = 1;
}

// exclusive scan in one block (len <= a few million); total to *tot
__global__ void k_scan_total(int* a, int len, int* tot) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (len + blockDim.x - 1) / blockDim.x;
  const int b = t * per, e = min(len, b + per);
  int s = 0;
  for (int i = b; i < e; ++i) s += a[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) { const int v = part[i]; part[i] = run; run += v; }
    *tot = run;
  }
  __syncthreads();
  int run = part[t];
  for (int i = b; i < e; ++i) { const int v = a[i]; a[i] = run; run += v; }
}

// ---------------------------------------------------------------------------
// level restriction
// ---------------------------------------------------------------------------

// the box containing level-l cell (x, y, z): the first box that exists
// walking up from level l, or -1
__device__ __forceinline__ int first_box_up(DHash H, int l, int64_t x, int64_t y, int64_t z,
                                            int& lev) {
  for (int lp = l; lp >= 0; --lp) {
    const int sh = l - lp;
    const int j = hash_find(H, loc_code(lp, (uint64_t)(x >> sh), (uint64_t)(y >> sh),
                                        (uint64_t)(z >> sh)));
    if (j >= 0) {
      lev = lp;
      return j;
    }
  }
  lev = -1;
  return -1;
}

// every leaf marks the leaves two or more levels coarser that touch it
__global__ void k_balance_mark(DBoxes B, DHash H, int nbox, int* nmarked) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbox || B.nkids[i] != 0) return;
  const int l = B.lvl[i];
  if (l < 2) return;
  int64_t x, y, z;
  cell_of(B.code[i], l, x, y, z);
  const int64_t side = (int64_t)1 << l;
  for (int d = 0; d < 27; ++d) {
    if (d == 13) continue;
    const int64_t nx = x + d % 3 - 1, ny = y + (d / 3) % 3 - 1, nz = z + d / 9 - 1;
    if (nx < 0 || ny < 0 || nz < 0 || nx >= side || ny >= side || nz >= side) continue;
    int lev;
    const int j = first_box_up(H, l, nx, ny, nz, lev);
    if (j < 0 || B.nkids[j] != 0 || lev > l - 2 || lev >= 20) continue;
    if (atomicExch(&B.mark[j], 1) == 0) atomicAdd(nmarked, 1);
  }
}

// split the marked leaves: children appended at an atomic counter (ids are
// renumbered canonically afterwards)
__global__ void k_balance_split(DBoxes B, DHash H, const uint64_t* __restrict__ keys, int nbox,
                                int* counter, int cap, int* fail) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbox || !B.mark[i]) return;
  B.mark[i] = 0;
  int cs[9], oc[8];
  const int c = octant_ranges(keys, B.start[i], B.end[i], B.lvl[i], cs, oc);
  const int base = atomicAdd(counter, c);
  if (base + c > cap) {
    *fail = 2;
    return;
  }
  if (!write_children(B, H, keys, i, base)) *fail = 1;
}

// ---------------------------------------------------------------------------
// canonical order (level, first point)
// ---------------------------------------------------------------------------

__global__ void k_order_keys(const DBoxes B, int nbox, uint64_t* k, int* v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbox) return;
  k[i] = ((uint64_t)B.lvl[i] << 32) | (uint64_t)(uint32_t)B.start[i];
  v[i] = i;
}

__global__ void k_inverse(const int* __restrict__ ord, int nbox, int* inv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nbox) inv[ord[t]] = t;
}

// out[t] = in[ord[t]] for every array; parents renumbered; first child by
// atomicMin (children of one box are consecutive in the new order)
__global__ void k_reorder(const DBoxes in, DBoxes out, const int* __restrict__ ord,
                          const int* __restrict__ inv, int nbox) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nbox) return;
  const int o = ord[t];
  out.lvl[t] = in.lvl[o];
  out.code[t] = in.code[o];
  out.start[t] = in.start[o];
  out.end[t] = in.end[o];
  out.nkids[t] = in.nkids[o];
  out.mark[t] = 0;
  const int p = in.parent[o];
  out.parent[t] = p >= 0 ? inv[p] : -1;
  if (p >= 0) atomicMin(&out.first_kid[inv[p]], t);
}

__global__ void k_hash_all(DBoxes B, DHash H, int nbox, int* fail) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nbox && !hash_insert(H, B.code[t], t)) *fail = 1;
}

// ---------------------------------------------------------------------------
// near and Q lists, same-level conflicts, coarse-leaf users
// ---------------------------------------------------------------------------

constexpr int kMaxCand = 125;

__device__ __forceinline__ int64_t dbox_gap(int la, int64_t ax, int64_t ay, int64_t az, int lb,
                                            int64_t bx, int64_t by, int64_t bz) {
  const int64_t ca[3] = {ax, ay, az}, cb[3] = {bx, by, bz};
  int64_t g = 0;
  for (int d = 0; d < 3; ++d) {
    const int64_t lo1 = ca[d] << (21 - la), hi1 = (ca[d] + 1) << (21 - la);
    const int64_t lo2 = cb[d] << (21 - lb), hi2 = (cb[d] + 1) << (21 - lb);
    const int64_t gd = max((int64_t)0, max(lo2 - hi1, lo1 - hi2));
    g = max(g, gd);
  }
  return g;
}

struct DLists {
  int* ncnt;   int* noff;   int* nlist;    // near boxes (ids), by first point
  int* qcnt;   int* qoff;   int* qlist;    // Q boxes
  int* scnt;   int* soff;   int* slist;    // same-level boxes at gap <= h
  int* ucnt;   int* uoff;                  // near boxes of coarser levels
  unsigned long long* ukey; int* uval;     // (level << 32 | coarse box) -> level box
};

// one thread per box of level >= 2 (ids t0 .. nbox - 1); fill = 0 counts,
// fill = 1 writes the lists at the scanned offsets
__global__ void __launch_bounds__(128) k_lists(DBoxes B, DHash H, int t0, int nbox, DLists Ls,
                                               int fill) {
  const int t = t0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nbox) return;
  const int l = B.lvl[t];
  int64_t x, y, z;
  cell_of(B.code[t], l, x, y, z);
  const int64_t side = (int64_t)1 << l, h = (int64_t)1 << (21 - l);
  int cand[kMaxCand], cst[kMaxCand];
  int nc = 0;
  for (int dz = -2; dz <= 2; ++dz)
    for (int dy = -2; dy <= 2; ++dy)
      for (int dx = -2; dx <= 2; ++dx) {
        const int64_t cx = x + dx, cy = y + dy, cz = z + dz;
        if (cx < 0 || cy < 0 || cz < 0 || cx >= side || cy >= side || cz >= side) continue;
        int lev;
        const int j = first_box_up(H, l, cx, cy, cz, lev);
        if (j < 0 || j == t) continue;
        if (lev != l && B.nkids[j] != 0) continue;   // refined but empty region
        // insert by first point, skipping duplicates (a coarse leaf covers
        // several cells)
        const int sj = B.start[j];
        int p = nc;
        bool dup = false;
        for (int q = 0; q < nc; ++q)
          if (cand[q] == j) { dup = true; break; }
        if (dup) continue;
        while (p > 0 && cst[p - 1] > sj) {
          cand[p] = cand[p - 1];
          cst[p] = cst[p - 1];
          --p;
        }
        cand[p] = j;
        cst[p] = sj;
        ++nc;
      }
  const int r = t - t0;
  int nn = 0, nq = 0, ns = 0, nu = 0;
  for (int q = 0; q < nc; ++q) {
    const int c = cand[q];
    const int lc = B.lvl[c];
    int64_t bx, by, bz;
    cell_of(B.code[c], lc, bx, by, bz);
    const int64_t g = dbox_gap(l, x, y, z, lc, bx, by, bz);
    if (g == 0) {
      if (fill) Ls.nlist[Ls.noff[r] + nn] = c;
      ++nn;
      if (lc < l) {
        if (fill) {
          Ls.ukey[Ls.uoff[r] + nu] = ((unsigned long long)l << 32) | (unsigned)c;
          Ls.uval[Ls.uoff[r] + nu] = t;
        }
        ++nu;
      }
    } else if (g <= h) {
      if (fill) Ls.qlist[Ls.qoff[r] + nq] = c;
      ++nq;
    }
    if (g <= h && lc == l) {
      if (fill) Ls.slist[Ls.soff[r] + ns] = c;
      ++ns;
    }
  }
  if (!fill) {
    Ls.ncnt[r] = nn;
    Ls.qcnt[r] = nq;
    Ls.scnt[r] = ns;
    Ls.ucnt[r] = nu;
  }
}

// ---------------------------------------------------------------------------
// colours: one warp per level walks the level's boxes in Morton order
// ---------------------------------------------------------------------------

constexpr int kMaxColours = 1024;

// first index in [a, b) of ukey with key >= k
__device__ __forceinline__ int lower_key(const unsigned long long* __restrict__ ukey, int a, int b,
                                         unsigned long long k) {
  while (a < b) {
    const int m = (a + b) >> 1;
    if (ukey[m] < k) a = m + 1; else b = m;
  }
  return a;
}

// Earlier conflicting boxes of every level box (one thread per box): the
// same-level boxes at gap <= h and the boxes sharing a coarser near leaf,
// each with an index below the box's own. fill = 0 counts, 1 writes.
__global__ void k_conflicts(const DBoxes B, const DLists Ls, int t0, int nbox, int nu_total,
                            int* ccnt, const int* coff, int* conf, int fill) {
  const int t = t0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nbox) return;
  const int r = t - t0;
  const int level = B.lvl[t];
  int c = 0;
  const int o0 = fill ? coff[r] : 0;
  for (int q = 0; q < Ls.scnt[r]; ++q) {
    const int o = Ls.slist[Ls.soff[r] + q];
    if (o < t) {
      if (fill) conf[o0 + c] = o;
      ++c;
    }
  }
  for (int q = 0; q < Ls.ncnt[r]; ++q) {
    const int cbox = Ls.nlist[Ls.noff[r] + q];
    if (B.lvl[cbox] >= level) continue;
    const unsigned long long key = ((unsigned long long)level << 32) | (unsigned)cbox;
    for (int u = lower_key(Ls.ukey, 0, nu_total, key); u < nu_total && Ls.ukey[u] == key; ++u) {
      const int o = Ls.uval[u];
      if (o < t) {
        if (fill) conf[o0 + c] = o;
        ++c;
      }
    }
  }
  if (!fill) ccnt[r] = c;
}

// Greedy colours in Morton order: one warp per level (level = lev0 +
// blockIdx.x, boxes [lstart[level], lstart[level + 1])) walks its boxes in
// order; a box takes the smallest colour that none of its earlier
// conflicting boxes has. Colours below 64 are gathered in registers and
// or-reduced over the warp, larger ones in a shared bit set. The next box's
// first 64 conflicts are loaded while the current box is coloured. Colours
// live in shared memory when the level fits (smem_boxes), else in col.
__global__ void __launch_bounds__(32) k_colour(const int* __restrict__ ccnt,
                                               const int* __restrict__ coff,
                                               const int* __restrict__ conf, const int* lstart,
                                               int lev0, int t0, int smem_boxes, int* col,
                                               int* ncol, int* fail) {
  extern __shared__ unsigned short scol[];
  __shared__ unsigned mask_hi[kMaxColours / 32];
  const int level = lev0 + blockIdx.x;
  const int b0 = lstart[level], b1 = lstart[level + 1];
  const int nb = b1 - b0;
  const int lane = threadIdx.x;
  const bool in_smem = nb <= smem_boxes;
  for (int w = lane; w < kMaxColours / 32; w += 32) mask_hi[w] = 0;
  __syncwarp();
  auto colour_of = [&](int o) -> int {
    return in_smem ? (int)scol[o - b0] : ((volatile int*)col)[o];
  };
  auto fetch = [&](int rb, int& cnt, int& e0, int& e1) {
    cnt = 0; e0 = -1; e1 = -1;
    if (rb >= b1) return;
    const int r = rb - t0;
    cnt = ccnt[r];
    const int off = coff[r];
    if (lane < cnt) e0 = conf[off + lane];
    if (lane + 32 < cnt) e1 = conf[off + 32 + lane];
  };
  int cnt, e0, e1;
  fetch(b0, cnt, e0, e1);
  int maxc = -1;
  for (int rb = b0; rb < b1; ++rb) {
    int ncnt, n0, n1;
    fetch(rb + 1, ncnt, n0, n1);   // independent of the colours: overlaps
    unsigned long long bits = 0;
    bool high = false;
    auto take = [&](int o) {
      const int c = colour_of(o);
      if (c < 64) bits |= 1ull << c;
      else { atomicOr(&mask_hi[c >> 5], 1u << (c & 31)); high = true; }
    };
    if (e0 >= 0) take(e0);
    if (e1 >= 0) take(e1);
    if (cnt > 64) {
      const int off = coff[rb - t0];
      for (int q = 64 + lane; q < cnt; q += 32) take(conf[off + q]);
    }
    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)bits);
    const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(bits >> 32));
    const bool any_high = __any_sync(0xffffffffu, high);
    __syncwarp();
    int c;
    if (lo != 0xffffffffu) c = __ffs(~lo) - 1;
    else if (hi != 0xffffffffu) c = 32 + __ffs(~hi) - 1;
    else {
      // every colour below 64 is taken: the shared set holds the rest
      const unsigned wv = lane >= 2 ? mask_hi[lane] : 0xffffffffu;
      const unsigned free_w = __ballot_sync(0xffffffffu, wv != 0xffffffffu);
      const int wf = free_w ? __ffs(free_w) - 1 : -1;
      const unsigned wsel = __shfl_sync(0xffffffffu, wv, wf < 0 ? 0 : wf);
      c = wf < 0 ? kMaxColours : wf * 32 + (__ffs(~wsel) - 1);
    }
    if (lane == 0) {
      if (c >= kMaxColours) *fail = 3;
      const int cc = c >= kMaxColours ? 0 : c;
      if (in_smem) scol[rb - b0] = (unsigned short)cc;
      ((volatile int*)col)[rb] = cc;
    }
    maxc = max(maxc, c);
    if (any_high) {
      mask_hi[lane] = 0;
    }
    __syncwarp();
    cnt = ncnt; e0 = n0; e1 = n1;
  }
  if (lane == 0) ncol[level] = maxc + 1;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

struct TreeFail {
  int code;
  std::string msg;
};

#define TCK(x)                                                                             \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess)                                                                 \
      throw TreeFail{e_ == cudaErrorMemoryAllocation ? -2 : -3,                            \
                     std::string(#x) + ": " + cudaGetErrorString(e_)};                     \
  } while (0)

// device allocations freed together
struct DMem {
  std::vector<void*> ptrs;
  template <class T>
  T* get(size_t count) {
    void* p = nullptr;
    TCK(cudaMalloc(&p, std::max<size_t>(1, count) * sizeof(T)));
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  void release(void* p) {
    auto it = std::find(ptrs.begin(), ptrs.end(), p);
    if (it != ptrs.end()) { cudaFree(p); ptrs.erase(it); }
  }
  void keep(void* p) {   // hand ownership to the caller
    auto it = std::find(ptrs.begin(), ptrs.end(), p);
    if (it != ptrs.end()) ptrs.erase(it);
  }
  ~DMem() { for (void* p : ptrs) cudaFree(p); }
};

template <class T>
std::vector<T> down(const T* d, size_t count, cudaStream_t st) {
  std::vector<T> h(count);
  if (count) TCK(cudaMemcpyAsync(h.data(), d, count * sizeof(T), cudaMemcpyDeviceToHost, st));
  TCK(cudaStreamSynchronize(st));
  return h;
}

int dgrid(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

// stable LSD radix sort of (key, value) pairs over the low 4 * passes bits;
// returns the buffers holding the result (k0/v0 or k1/v1)
std::pair<uint64_t*, int*> radix_sort(uint64_t* k0, int* v0, uint64_t* k1, int* v1, DMem& mem,
                                      int64_t n, int passes, cudaStream_t st) {
  if (n <= 0) return {k0, v0};
  const int nblk = (int)((n + kSortTile - 1) / kSortTile);
  int* hist = mem.get<int>(16 * (size_t)nblk);
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = 4 * pass;
    FMMLU_LAUNCH("radix_hist", st,
                 k_radix_hist<<<nblk, kSortThreads, 0, st>>>(k0, n, shift, hist, nblk));
    FMMLU_LAUNCH("radix_scan", st, k_scan_small<<<1, 1024, 0, st>>>(hist, 16 * nblk));
    FMMLU_LAUNCH("radix_scatter", st,
                 k_radix_scatter<<<nblk, kSortThreads, 0, st>>>(k0, v0, n, shift, hist, nblk, k1,
                                                                v1));
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  return {k0, v0};
}

// growable box arrays plus their hash table
struct BoxStore {
  DMem mem;
  DBoxes B{};
  DHash H{};
  int cap = 0;
  void alloc(int c, cudaStream_t st) {
    DBoxes nb;
    nb.lvl = mem.get<int>(c);
    nb.code = mem.get<unsigned long long>(c);
    nb.start = mem.get<int>(c);
    nb.end = mem.get<int>(c);
    nb.parent = mem.get<int>(c);
    nb.nkids = mem.get<int>(c);
    nb.mark = mem.get<int>(c);
    nb.first_kid = mem.get<int>(c);
    TCK(cudaMemsetAsync(nb.mark, 0, sizeof(int) * (size_t)c, st));
    B = nb;
    cap = c;
    uint32_t hc = 1024;
    while (hc < 2u * (uint32_t)c) hc <<= 1;
    H.keys = mem.get<unsigned long long>(hc);
    H.vals = mem.get<int>(hc);
    H.mask = hc - 1;
    TCK(cudaMemsetAsync(H.keys, 0, sizeof(unsigned long long) * hc, st));
  }
  // at least `need` boxes; the first `used` are kept and rehashed
  void ensure(int need, int used, int* d_fail, cudaStream_t st) {
    if (need <= cap) return;
    DBoxes old = B;
    DHash oh = H;
    const int oc = cap;
    alloc(std::max(need, 2 * oc), st);
    auto cp = [&](void* dst, const void* src, size_t bytes) {
      if (bytes) TCK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
    };
    cp(B.lvl, old.lvl, 4 * (size_t)used);
    cp(B.code, old.code, 8 * (size_t)used);
    cp(B.start, old.start, 4 * (size_t)used);
    cp(B.end, old.end, 4 * (size_t)used);
    cp(B.parent, old.parent, 4 * (size_t)used);
    cp(B.nkids, old.nkids, 4 * (size_t)used);
    cp(B.mark, old.mark, 4 * (size_t)used);
    if (used > 0)
      FMMLU_LAUNCH("tree_hash", st,
                   k_hash_all<<<dgrid(used, 256), 256, 0, st>>>(B, H, used, d_fail));
    TCK(cudaStreamSynchronize(st));
    for (void* p : {(void*)old.lvl, (void*)old.code, (void*)old.start, (void*)old.end,
                    (void*)old.parent, (void*)old.nkids, (void*)old.mark, (void*)old.first_kid,
                    (void*)oh.keys, (void*)oh.vals})
      mem.release(p);
  }
};

__global__ void k_root(DBoxes B, DHash H, int n, int* fail) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  B.lvl[0] = 0;
  B.code[0] = 1ull;
  B.start[0] = 0;
  B.end[0] = n;
  B.parent[0] = -1;
  B.nkids[0] = 0;
  B.mark[0] = 0;
  if (!hash_insert(H, 1ull, 0)) *fail = 1;
}

}  // namespace

int gpu_build_tree(const double* pts, int64_t n, int leaf_size, TreeHost& T, int** d_perm_out,
                   std::string& msg, int verbose, cudaStream_t st) {
  const auto t_start = std::chrono::steady_clock::now();
  std::vector<std::pair<const char*, double>> phases;
  auto phase = [&](const char* name) {
    if (!verbose) return;
    TCK(cudaStreamSynchronize(st));
    phases.push_back({name, std::chrono::duration<double, std::milli>(
                                std::chrono::steady_clock::now() - t_start).count()});
  };
  try {
    DMem mem;
    int* d_flags = mem.get<int>(8);   // [0] hash/fail, [1] bad point, [2] counter, [3] total
    TCK(cudaMemsetAsync(d_flags, 0, 8 * sizeof(int), st));
    // 1. bounding cube from exact extrema (the same arithmetic as the oracle)
    const int eb = (int)std::min<int64_t>(1024, (n + kBoxThreads - 1) / kBoxThreads);
    double* d_ext = mem.get<double>(6 * (size_t)eb);
    FMMLU_LAUNCH("tree_extrema", st,
                 k_extrema<<<eb, kBoxThreads, 0, st>>>(pts, n, d_ext, d_flags + 1));
    FMMLU_LAUNCH("tree_extrema", st, k_extrema_final<<<1, 32, 0, st>>>(d_ext, eb));
    std::vector<double> ext = down(d_ext, 6, st);
    if (down(d_flags + 1, 1, st)[0]) throw TreeFail{-1, "non-finite point coordinate"};
    double extent = 0, center[3];
    for (int a = 0; a < 3; ++a) {
      center[a] = (ext[a] + ext[3 + a]) / 2.0;
      extent = std::max(extent, ext[3 + a] - ext[a]);
    }
    double side = extent * (1.0 + 1e-12);
    if (!(side > 0.0)) side = 1.0;
    T.n = n;
    T.side = side;
    for (int a = 0; a < 3; ++a) T.corner[a] = center[a] - side / 2.0;
    T.leaf_size = leaf_size;
    // Morton keys, sorted with the point indices
    uint64_t* k0 = mem.get<uint64_t>(n);
    uint64_t* k1 = mem.get<uint64_t>(n);
    int* v0 = mem.get<int>(n);
    int* v1 = mem.get<int>(n);
    FMMLU_LAUNCH("morton", st, k_morton<<<dgrid(n, 256), 256, 0, st>>>(
                                   pts, n, T.corner[0], T.corner[1], T.corner[2], side, k0, v0));
    auto sorted = radix_sort(k0, v0, k1, v1, mem, n, 16, st);
    phase("keys");
    const uint64_t* keys = sorted.first;
    int* d_perm = sorted.second;
    // 2. hierarchy
    BoxStore S;
    S.alloc((int)std::max<int64_t>(1024, 4 * n / std::max(1, leaf_size)), st);
    FMMLU_LAUNCH("tree_root", st, k_root<<<1, 1, 0, st>>>(S.B, S.H, (int)n, d_flags));
    int b0 = 0, b1 = 1;
    int* d_cnt = mem.get<int>((size_t)n + 1);
    while (b1 > b0) {
      const int nl = b1 - b0;
      FMMLU_LAUNCH("tree_split", st, k_child_count<<<dgrid(nl, 128), 128, 0, st>>>(
                                         S.B, keys, b0, b1, leaf_size, d_cnt));
      FMMLU_LAUNCH("tree_scan", st, k_scan_total<<<1, 1024, 0, st>>>(d_cnt, nl, d_flags + 3));
      const int tot = down(d_flags + 3, 1, st)[0];
      if (tot == 0) break;
      S.ensure(b1 + tot, b1, d_flags, st);
      FMMLU_LAUNCH("tree_split", st, k_child_write<<<dgrid(nl, 128), 128, 0, st>>>(
                                         S.B, S.H, keys, b0, b1, leaf_size, d_cnt, b1, d_flags));
      b0 = b1;
      b1 += tot;
    }
    int nbox = b1;
    phase("hierarchy");
    // 3. level restriction, in rounds
    for (;;) {
      TCK(cudaMemsetAsync(d_flags + 2, 0, sizeof(int), st));
      FMMLU_LAUNCH("tree_balance", st, k_balance_mark<<<dgrid(nbox, 128), 128, 0, st>>>(
                                           S.B, S.H, nbox, d_flags + 2));
      const int marked = down(d_flags + 2, 1, st)[0];
      if (marked == 0) break;
      S.ensure(nbox + 8 * marked, nbox, d_flags, st);
      TCK(cudaMemcpyAsync(d_flags + 2, &nbox, sizeof(int), cudaMemcpyHostToDevice, st));
      FMMLU_LAUNCH("tree_balance", st, k_balance_split<<<dgrid(nbox, 128), 128, 0, st>>>(
                                           S.B, S.H, keys, nbox, d_flags + 2, S.cap, d_flags));
      nbox = down(d_flags + 2, 1, st)[0];
    }
    if (int f = down(d_flags, 1, st)[0]) throw TreeFail{-3, "tree construction overflow " + std::to_string(f)};
    phase("balance");
    // 4. canonical ids: (level, first point)
    uint64_t* ok0 = mem.get<uint64_t>(nbox);
    uint64_t* ok1 = mem.get<uint64_t>(nbox);
    int* ov0 = mem.get<int>(nbox);
    int* ov1 = mem.get<int>(nbox);
    FMMLU_LAUNCH("tree_order", st, k_order_keys<<<dgrid(nbox, 256), 256, 0, st>>>(S.B, nbox, ok0, ov0));
    const int* ord = radix_sort(ok0, ov0, ok1, ov1, mem, nbox, 10, st).second;
    int* inv = mem.get<int>(nbox);
    FMMLU_LAUNCH("tree_order", st, k_inverse<<<dgrid(nbox, 256), 256, 0, st>>>(ord, nbox, inv));
    BoxStore C;
    C.alloc(nbox, st);
    TCK(cudaMemsetAsync(C.B.first_kid, 0x7f, sizeof(int) * (size_t)nbox, st));
    FMMLU_LAUNCH("tree_order", st, k_reorder<<<dgrid(nbox, 256), 256, 0, st>>>(S.B, C.B, ord, inv, nbox));
    FMMLU_LAUNCH("tree_hash", st, k_hash_all<<<dgrid(nbox, 256), 256, 0, st>>>(C.B, C.H, nbox, d_flags));
    const DBoxes& B = C.B;
    std::vector<int> lvl = down(B.lvl, nbox, st);
    int nlevels = lvl.back() + 1;
    std::vector<int> lstart(nlevels + 2, nbox);
    for (int t = nbox - 1; t >= 0; --t) lstart[lvl[t]] = t;
    for (int l = nlevels - 1; l >= 0; --l) lstart[l] = std::min(lstart[l], lstart[l + 1]);
    T.nlevels = nlevels;
    phase("ids");
    // 5. near / Q lists and conflicts of every box of level >= 2
    const int t0 = nlevels > 2 ? lstart[2] : nbox;
    const int nb2 = nbox - t0;
    DLists Ls{};
    std::vector<int> ncol(nlevels + 1, 0), col;
    std::vector<int> h_noff, h_ncnt, h_nlist, h_qoff, h_qcnt, h_qlist;
    if (nb2 > 0) {
      int* cnts = mem.get<int>(8 * (size_t)nb2);
      Ls.ncnt = cnts; Ls.qcnt = cnts + nb2; Ls.scnt = cnts + 2 * nb2; Ls.ucnt = cnts + 3 * nb2;
      Ls.noff = cnts + 4 * nb2; Ls.qoff = cnts + 5 * nb2; Ls.soff = cnts + 6 * nb2;
      Ls.uoff = cnts + 7 * nb2;
      FMMLU_LAUNCH("tree_lists", st, k_lists<<<dgrid(nb2, 128), 128, 0, st>>>(
                                         B, C.H, t0, nbox, Ls, 0));
      TCK(cudaMemcpyAsync(Ls.noff, Ls.ncnt, 4 * sizeof(int) * (size_t)nb2,
                          cudaMemcpyDeviceToDevice, st));
      int tot[4];
      for (int q = 0; q < 4; ++q) {
        FMMLU_LAUNCH("tree_scan", st,
                     k_scan_total<<<1, 1024, 0, st>>>(cnts + (4 + q) * (size_t)nb2, nb2, d_flags + 4 + q));
      }
      std::vector<int> tv = down(d_flags + 4, 4, st);
      for (int q = 0; q < 4; ++q) tot[q] = tv[q];
      Ls.nlist = mem.get<int>(tot[0]);
      Ls.qlist = mem.get<int>(tot[1]);
      Ls.slist = mem.get<int>(tot[2]);
      unsigned long long* uk0 = mem.get<unsigned long long>(tot[3]);
      unsigned long long* uk1 = mem.get<unsigned long long>(tot[3]);
      int* uv0 = mem.get<int>(tot[3]);
      int* uv1 = mem.get<int>(tot[3]);
      Ls.ukey = uk0;
      Ls.uval = uv0;
      FMMLU_LAUNCH("tree_lists", st, k_lists<<<dgrid(nb2, 128), 128, 0, st>>>(
                                         B, C.H, t0, nbox, Ls, 1));
      auto us = radix_sort(reinterpret_cast<uint64_t*>(uk0), uv0, reinterpret_cast<uint64_t*>(uk1),
                           uv1, mem, tot[3], 10, st);
      Ls.ukey = reinterpret_cast<unsigned long long*>(us.first);
      Ls.uval = us.second;
      phase("lists");
      // 6. colours, one warp per level
      int* d_col = mem.get<int>(nbox);
      int* d_ncol = mem.get<int>(nlevels + 1);
      TCK(cudaMemsetAsync(d_col, 0, sizeof(int) * (size_t)nbox, st));
      TCK(cudaMemsetAsync(d_ncol, 0, sizeof(int) * (size_t)(nlevels + 1), st));
      int* d_lstart = mem.get<int>(nlevels + 2);
      TCK(cudaMemcpyAsync(d_lstart, lstart.data(), sizeof(int) * (nlevels + 2),
                          cudaMemcpyHostToDevice, st));
      int maxnb = 0;
      for (int l = 2; l < nlevels; ++l) maxnb = std::max(maxnb, lstart[l + 1] - lstart[l]);
      const int smem_boxes = maxnb <= 65536 ? maxnb : 0;
      const size_t csm = 2 * (size_t)smem_boxes;
      int* ccnt = mem.get<int>(nb2);
      int* coff = mem.get<int>(nb2);
      FMMLU_LAUNCH("tree_colour", st, k_conflicts<<<dgrid(nb2, 128), 128, 0, st>>>(
                                          B, Ls, t0, nbox, tot[3], ccnt, coff, nullptr, 0));
      TCK(cudaMemcpyAsync(coff, ccnt, sizeof(int) * (size_t)nb2, cudaMemcpyDeviceToDevice, st));
      FMMLU_LAUNCH("tree_scan", st, k_scan_total<<<1, 1024, 0, st>>>(coff, nb2, d_flags + 2));
      const int nconf = down(d_flags + 2, 1, st)[0];
      int* conf = mem.get<int>(nconf);
      FMMLU_LAUNCH("tree_colour", st, k_conflicts<<<dgrid(nb2, 128), 128, 0, st>>>(
                                          B, Ls, t0, nbox, tot[3], ccnt, coff, conf, 1));
      TCK(cudaFuncSetAttribute(k_colour, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
      FMMLU_LAUNCH("tree_colour", st, k_colour<<<nlevels - 2, 32, csm, st>>>(
                                          ccnt, coff, conf, d_lstart, 2, t0, smem_boxes, d_col,
                                          d_ncol, d_flags));
      phase("colours");
      col = down(d_col, nbox, st);
      ncol = down(d_ncol, nlevels + 1, st);
      h_ncnt = down(Ls.ncnt, nb2, st);
      h_noff = down(Ls.noff, nb2, st);
      h_nlist = down(Ls.nlist, tot[0], st);
      h_qcnt = down(Ls.qcnt, nb2, st);
      h_qoff = down(Ls.qoff, nb2, st);
      h_qlist = down(Ls.qlist, tot[1], st);
      if (int f = down(d_flags, 1, st)[0])
        throw TreeFail{-3, "tree construction failed (" + std::to_string(f) + ")"};
    }
    // download the boxes into the host description
    std::vector<unsigned long long> code = down(B.code, nbox, st);
    std::vector<int> bs = down(B.start, nbox, st), be = down(B.end, nbox, st);
    std::vector<int> par = down(B.parent, nbox, st), nk = down(B.nkids, nbox, st);
    std::vector<int> fk = down(B.first_kid, nbox, st);
    T.boxes.assign(nbox, HBox());
    for (int t = 0; t < nbox; ++t) {
      HBox& b = T.boxes[t];
      const int l = lvl[t];
      const uint64_t m = code[t] & ((1ull << (3 * l)) - 1);
      b.level = l;
      b.cx = (int64_t)compact3(m);
      b.cy = (int64_t)compact3(m >> 1);
      b.cz = (int64_t)compact3(m >> 2);
      b.start = bs[t];
      b.end = be[t];
      b.parent = par[t];
      b.kids.resize(nk[t]);
      for (int c = 0; c < nk[t]; ++c) b.kids[c] = fk[t] + c;
    }
    T.perm = down(d_perm, n, st);
    T.levels.clear();
    // current boxes of every level: the level's boxes merged by first point
    // with the leaves of coarser levels
    std::vector<int> coarse;   // leaves of levels < l, by first point
    for (int l = 0; l < nlevels; ++l) {
      std::vector<int> lev(lstart[l + 1] - lstart[l]);
      std::iota(lev.begin(), lev.end(), lstart[l]);
      if (l >= 2) {
        HLevel L;
        L.level = l;
        L.boxes = lev;
        L.current.resize(coarse.size() + lev.size());
        std::merge(coarse.begin(), coarse.end(), lev.begin(), lev.end(), L.current.begin(),
                   [&](int a, int b) { return T.boxes[a].start < T.boxes[b].start; });
        const int nb = (int)lev.size();
        L.nbeg.resize(nb); L.ncnt.resize(nb); L.qbeg.resize(nb); L.qcnt.resize(nb);
        L.colour.resize(nb);
        for (int r = 0; r < nb; ++r) {
          const int i = lstart[l] + r - t0;
          L.nbeg[r] = (int)L.nlist.size();
          L.ncnt[r] = h_ncnt[i];
          L.nlist.insert(L.nlist.end(), h_nlist.begin() + h_noff[i],
                         h_nlist.begin() + h_noff[i] + h_ncnt[i]);
          L.qbeg[r] = (int)L.qlist.size();
          L.qcnt[r] = h_qcnt[i];
          L.qlist.insert(L.qlist.end(), h_qlist.begin() + h_qoff[i],
                         h_qlist.begin() + h_qoff[i] + h_qcnt[i]);
          L.colour[r] = col[lstart[l] + r];
        }
        L.ncolours = ncol[l];
        L.order.resize(nb);
        std::iota(L.order.begin(), L.order.end(), 0);
        std::stable_sort(L.order.begin(), L.order.end(),
                         [&](int a, int b) { return L.colour[a] < L.colour[b]; });
        T.levels[l] = std::move(L);
      }
      std::vector<int> leaves;
      for (int t : lev)
        if (T.boxes[t].kids.empty()) leaves.push_back(t);
      std::vector<int> merged(coarse.size() + leaves.size());
      std::merge(coarse.begin(), coarse.end(), leaves.begin(), leaves.end(), merged.begin(),
                 [&](int a, int b) { return T.boxes[a].start < T.boxes[b].start; });
      coarse.swap(merged);
    }
    phase("host description");
    if (verbose) {
      std::fprintf(stderr, "[fmmlu] tree: %d boxes, %d levels;", nbox, nlevels);
      for (auto& p : phases) std::fprintf(stderr, " %s %.2f ms", p.first, p.second);
      std::fprintf(stderr, "\n");
    }
    // the sorted permutation stays on the device for the factorization
    int* keep = mem.get<int>(n);
    TCK(cudaMemcpyAsync(keep, d_perm, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    TCK(cudaStreamSynchronize(st));
    mem.keep(keep);
    *d_perm_out = keep;
    return 0;
  } catch (const TreeFail& f) {
    msg = f.msg;
    return f.code;
  }
}

// current boxes of a level (its boxes plus coarser leaves), by first point
std::vector<int> current_boxes(const TreeHost& T, int level) {
  auto it = T.levels.find(level);
  if (it != T.levels.end()) return it->second.current;
  std::vector<int> cur;
  for (int i = 0; i < (int)T.boxes.size(); ++i) {
    const HBox& b = T.boxes[i];
    if (b.level == level || (b.kids.empty() && b.level < level)) cur.push_back(i);
  }
  std::sort(cur.begin(), cur.end(), [&](int a, int b) { return T.boxes[a].start < T.boxes[b].start; });
  return cur;
}

}  // namespace fmmlu
