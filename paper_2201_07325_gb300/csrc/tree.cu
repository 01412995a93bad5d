// Octree construction (Sec. 4 preamble, Sec. 4.3).
//
// GPU: integer coordinates q = floor((x - corner)/side * 2^21) (clipped to
// [0, 2^21 - 1]), 63-bit Morton keys (bit 3b <- x_b, 3b+1 <- y_b, 3b+2 <- z_b),
// and a stable LSD radix sort of (key, index) pairs, so equal keys keep the
// input order.
//
// Host (from the sorted keys): boxes are split while they hold more than s
// points (depth cap 21, empty children dropped); then the level restriction of
// Sec. 4 -- a leaf touching (face, edge or corner) a leaf two or more levels
// finer is split -- is applied until nothing changes (the minimal balanced
// refinement, unique whatever the order of splits). Box ids are ordered by
// (level, Morton). For every level l >= 2 the current boxes are the level-l
// boxes plus all coarser leaves; N(B) = current boxes touching B; Q(B) =
// current boxes at max-norm gap in (0, h_l]; colours are greedy in Morton
// order over the conflict relation gap <= h_l or shared closed neighbourhood.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <unordered_map>
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

#define TRY(x)                                   \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_ != cudaSuccess) return (int)e_;       \
  } while (0)

int gpu_morton_sort(const double* pts, int64_t n, const double corner[3], double side,
                    uint64_t* keys_host, int* perm_host, cudaStream_t st) {
  uint64_t *k0 = nullptr, *k1 = nullptr;
  int *v0 = nullptr, *v1 = nullptr, *hist = nullptr;
  int nblk = (int)((n + kSortTile - 1) / kSortTile);
  int rc = 0;
  do {
    if ((rc = (int)cudaMalloc(&k0, n * 8))) break;
    if ((rc = (int)cudaMalloc(&k1, n * 8))) break;
    if ((rc = (int)cudaMalloc(&v0, n * 4))) break;
    if ((rc = (int)cudaMalloc(&v1, n * 4))) break;
    if ((rc = (int)cudaMalloc(&hist, (size_t)16 * nblk * 4))) break;
    FMMLU_LAUNCH("morton", st, k_morton<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                                      pts, n, corner[0], corner[1], corner[2], side, k0, v0));
    for (int pass = 0; pass < 16; ++pass) {
      int shift = 4 * pass;
      FMMLU_LAUNCH("radix_hist", st, k_radix_hist<<<nblk, kSortThreads, 0, st>>>(k0, n, shift, hist, nblk));
      FMMLU_LAUNCH("radix_scan", st, k_scan_small<<<1, 1024, 0, st>>>(hist, 16 * nblk));
      FMMLU_LAUNCH("radix_scatter", st, k_radix_scatter<<<nblk, kSortThreads, 0, st>>>(
                                             k0, v0, n, shift, hist, nblk, k1, v1));
      std::swap(k0, k1);
      std::swap(v0, v1);
    }
    if ((rc = (int)cudaGetLastError())) break;
    if ((rc = (int)cudaMemcpyAsync(keys_host, k0, n * 8, cudaMemcpyDeviceToHost, st))) break;
    if ((rc = (int)cudaMemcpyAsync(perm_host, v0, n * 4, cudaMemcpyDeviceToHost, st))) break;
    rc = (int)cudaStreamSynchronize(st);
  } while (0);
  cudaFree(k0); cudaFree(k1); cudaFree(v0); cudaFree(v1); cudaFree(hist);
  return rc;
}

// ---------------------------------------------------------------------------
// host: hierarchy, level restriction, lists, colouring
// ---------------------------------------------------------------------------

static inline uint64_t cell_key(int level, int64_t cx, int64_t cy, int64_t cz) {
  return ((uint64_t)level << 58) ^ ((uint64_t)cx << 38) ^ ((uint64_t)cy << 19) ^ (uint64_t)cz;
}

uint64_t morton3_host(int64_t cx, int64_t cy, int64_t cz) {
  uint64_t k = 0;
  for (int b = 0; b < 21; ++b) {
    k |= (uint64_t)((cx >> b) & 1) << (3 * b);
    k |= (uint64_t)((cy >> b) & 1) << (3 * b + 1);
    k |= (uint64_t)((cz >> b) & 1) << (3 * b + 2);
  }
  return k;
}

// max-norm gap between closed boxes at the finest resolution
int64_t box_gap(const HBox& a, const HBox& b) {
  int64_t g = 0;
  int64_t ca[3] = {a.cx, a.cy, a.cz}, cb[3] = {b.cx, b.cy, b.cz};
  for (int d = 0; d < 3; ++d) {
    int64_t lo1 = ca[d] << (21 - a.level), hi1 = (ca[d] + 1) << (21 - a.level);
    int64_t lo2 = cb[d] << (21 - b.level), hi2 = (cb[d] + 1) << (21 - b.level);
    int64_t gd = std::max<int64_t>(0, std::max(lo2 - hi1, lo1 - hi2));
    g = std::max(g, gd);
  }
  return g;
}

static void split_node(std::vector<HBox>& nodes, int i, const std::vector<uint64_t>& keys) {
  HBox b = nodes[i];
  int l = b.level;
  int sh = 3 * (21 - l - 1);
  int64_t s = b.start;
  std::vector<int> kids;
  while (s < b.end) {
    int code = (int)((keys[s] >> sh) & 7);
    int64_t e = s + 1;
    while (e < b.end && (int)((keys[e] >> sh) & 7) == code) ++e;
    HBox c;
    c.level = l + 1;
    c.cx = 2 * b.cx + (code & 1);
    c.cy = 2 * b.cy + ((code >> 1) & 1);
    c.cz = 2 * b.cz + ((code >> 2) & 1);
    c.start = s; c.end = e; c.parent = i;
    nodes.push_back(c);
    kids.push_back((int)nodes.size() - 1);
    s = e;
  }
  nodes[i].kids = kids;
}

static bool any_leaf_touching(const std::vector<HBox>& nodes, int a, const HBox& L) {
  for (int c : nodes[a].kids) {
    if (box_gap(nodes[c], L) == 0) {
      if (nodes[c].kids.empty()) return true;
      if (any_leaf_touching(nodes, c, L)) return true;
    }
  }
  return false;
}

void build_host_tree(TreeHost& T, int leaf_size) {
  int64_t n = T.n;
  T.leaf_size = leaf_size;
  std::vector<HBox> nodes;
  HBox root;
  root.level = 0; root.cx = root.cy = root.cz = 0; root.start = 0; root.end = n; root.parent = -1;
  nodes.push_back(root);
  std::vector<int> work = {0};
  while (!work.empty()) {
    int i = work.back();
    work.pop_back();
    if (nodes[i].end - nodes[i].start > leaf_size && nodes[i].level < 21) {
      split_node(nodes, i, T.keys);
      for (int c : nodes[i].kids) work.push_back(c);
    }
  }
  // level restriction
  std::unordered_map<uint64_t, int> where;
  for (int i = 0; i < (int)nodes.size(); ++i)
    where[cell_key(nodes[i].level, nodes[i].cx, nodes[i].cy, nodes[i].cz)] = i;
  for (;;) {
    std::vector<int> todo;
    for (int i = 0; i < (int)nodes.size(); ++i) {
      const HBox& L = nodes[i];
      if (!L.kids.empty() || L.level >= 20) continue;
      int l1 = L.level + 1;
      int64_t side = (int64_t)1 << l1;
      bool need = false;
      for (int dz = -1; dz <= 2 && !need; ++dz)
        for (int dy = -1; dy <= 2 && !need; ++dy)
          for (int dx = -1; dx <= 2 && !need; ++dx) {
            if (dx >= 0 && dx <= 1 && dy >= 0 && dy <= 1 && dz >= 0 && dz <= 1) continue;
            int64_t x = 2 * L.cx + dx, y = 2 * L.cy + dy, z = 2 * L.cz + dz;
            if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) continue;
            auto it = where.find(cell_key(l1, x, y, z));
            if (it == where.end()) continue;
            if (nodes[it->second].kids.empty()) continue;
            if (any_leaf_touching(nodes, it->second, L)) need = true;
          }
      if (need) todo.push_back(i);
    }
    if (todo.empty()) break;
    for (int i : todo) {
      size_t before = nodes.size();
      split_node(nodes, i, T.keys);
      for (size_t c = before; c < nodes.size(); ++c)
        where[cell_key(nodes[c].level, nodes[c].cx, nodes[c].cy, nodes[c].cz)] = (int)c;
    }
  }
  // canonical ids by (level, Morton)
  std::vector<int> order(nodes.size());
  for (size_t i = 0; i < nodes.size(); ++i) order[i] = (int)i;
  std::vector<uint64_t> mk(nodes.size());
  for (size_t i = 0; i < nodes.size(); ++i) mk[i] = morton3_host(nodes[i].cx, nodes[i].cy, nodes[i].cz);
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (nodes[a].level != nodes[b].level) return nodes[a].level < nodes[b].level;
    return mk[a] < mk[b];
  });
  std::vector<int> remap(nodes.size());
  for (size_t i = 0; i < order.size(); ++i) remap[order[i]] = (int)i;
  T.boxes.assign(nodes.size(), HBox());
  T.nlevels = 0;
  for (size_t i = 0; i < order.size(); ++i) {
    HBox b = nodes[order[i]];
    b.parent = b.parent >= 0 ? remap[b.parent] : -1;
    for (int& c : b.kids) c = remap[c];
    std::sort(b.kids.begin(), b.kids.end());
    T.boxes[i] = b;
    T.nlevels = std::max(T.nlevels, b.level + 1);
  }
  T.where.clear();
  for (int i = 0; i < (int)T.boxes.size(); ++i)
    T.where[cell_key(T.boxes[i].level, T.boxes[i].cx, T.boxes[i].cy, T.boxes[i].cz)] = i;
  T.levels.clear();
  for (int l = 2; l < T.nlevels; ++l) T.levels[l] = build_level(T, l);
}

std::vector<int> current_boxes(const TreeHost& T, int level) {
  std::vector<int> cur;
  for (int i = 0; i < (int)T.boxes.size(); ++i) {
    const HBox& b = T.boxes[i];
    if (b.level == level || (b.kids.empty() && b.level < level)) cur.push_back(i);
  }
  std::sort(cur.begin(), cur.end(), [&](int a, int b) { return T.boxes[a].start < T.boxes[b].start; });
  return cur;
}

// current box at `level` containing level-`level` cell c, or -1 (empty region)
static int current_at(const TreeHost& T, int level, int64_t x, int64_t y, int64_t z) {
  for (int l = level; l >= 0; --l) {
    auto it = T.where.find(cell_key(l, x, y, z));
    if (it != T.where.end()) {
      const HBox& b = T.boxes[it->second];
      if (l == level || b.kids.empty()) return it->second;
      return -1;
    }
    x >>= 1; y >>= 1; z >>= 1;
  }
  return -1;
}

HLevel build_level(const TreeHost& T, int level) {
  HLevel L;
  L.level = level;
  for (int i = 0; i < (int)T.boxes.size(); ++i)
    if (T.boxes[i].level == level) L.boxes.push_back(i);
  L.current = current_boxes(T, level);
  int64_t h = (int64_t)1 << (21 - level);
  int64_t side = (int64_t)1 << level;
  int nb = (int)L.boxes.size();
  L.nbeg.resize(nb); L.ncnt.resize(nb); L.qbeg.resize(nb); L.qcnt.resize(nb);
  std::vector<std::vector<int>> samelevel(nb);   // level boxes with gap <= h
  std::unordered_map<int, int> pos_in_level;
  for (int r = 0; r < nb; ++r) pos_in_level[L.boxes[r]] = r;
  std::unordered_map<int, std::vector<int>> coarse_users;   // coarse leaf -> level boxes
  for (int r = 0; r < nb; ++r) {
    const HBox& B = T.boxes[L.boxes[r]];
    std::vector<int> cand;
    for (int dz = -2; dz <= 2; ++dz)
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
          int64_t x = B.cx + dx, y = B.cy + dy, z = B.cz + dz;
          if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) continue;
          int c = current_at(T, level, x, y, z);
          if (c >= 0 && c != L.boxes[r]) cand.push_back(c);
        }
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    std::sort(cand.begin(), cand.end(),
              [&](int a, int b) { return T.boxes[a].start < T.boxes[b].start; });
    L.nbeg[r] = (int)L.nlist.size();
    std::vector<int> q;
    for (int c : cand) {
      int64_t g = box_gap(B, T.boxes[c]);
      if (g == 0) {
        L.nlist.push_back(c);
        if (T.boxes[c].level < level) coarse_users[c].push_back(r);
      } else if (g <= h) {
        q.push_back(c);
      }
      if (g <= h && T.boxes[c].level == level) samelevel[r].push_back(pos_in_level[c]);
    }
    L.ncnt[r] = (int)L.nlist.size() - L.nbeg[r];
    L.qbeg[r] = (int)L.qlist.size();
    L.qlist.insert(L.qlist.end(), q.begin(), q.end());
    L.qcnt[r] = (int)q.size();
  }
  // greedy colouring in Morton (= id) order
  L.colour.assign(nb, -1);
  L.ncolours = 0;
  std::vector<int> mark;
  for (int r = 0; r < nb; ++r) {
    std::vector<int> conf = samelevel[r];
    for (int j = L.nbeg[r]; j < L.nbeg[r] + L.ncnt[r]; ++j) {
      int c = L.nlist[j];
      if (T.boxes[c].level < level) {
        const auto& u = coarse_users[c];
        conf.insert(conf.end(), u.begin(), u.end());
      }
    }
    mark.assign(L.ncolours + 2, 0);
    for (int o : conf)
      if (o < r && L.colour[o] >= 0) mark[L.colour[o]] = 1;
    int c = 0;
    while (mark[c]) ++c;
    L.colour[r] = c;
    L.ncolours = std::max(L.ncolours, c + 1);
  }
  L.order.resize(nb);
  for (int r = 0; r < nb; ++r) L.order[r] = r;
  std::stable_sort(L.order.begin(), L.order.end(),
                   [&](int a, int b) { return L.colour[a] < L.colour[b]; });
  return L;
}

}  // namespace fmmlu
