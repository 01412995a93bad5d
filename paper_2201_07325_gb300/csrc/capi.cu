// C ABI and host scheduler of the FMM-LU factorization.
//
// Factorization (Sec. 4.2, RS-S): levels from the finest up to level 2. At
// the start of a level the current boxes (level boxes plus coarser leaves)
// get their level-start active lists (a parent's = the concatenation of its
// children's skeletons), the Schur-update blocks of the previous level are
// gathered into blocks between the new current boxes (k_merge), and the
// per-box descriptors are uploaded. Boxes are then processed colour by
// colour; each colour is one launch per step (gather rows, assemble the ID
// matrix, CPQR + T, assemble the elimination blocks, the two X GEMMs, X_RR
// inverse, W GEMM and the scattered Schur update). After the level the host
// reads back the ranks and builds the next level. The stop rule of Sec. 4.2
// (no box with active far DOFs) and the root block elimination follow.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <set>
#include <sstream>
#include <stdexcept>
#include <thread>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/fmmlu.h"
#include "fmmlu_internal.h"
#include "prof.h"
#include "tree_host.h"

using namespace fmmlu;

namespace {

thread_local std::string g_err;

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define CK(x)                                                                              \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess)                                                                 \
      throw Error(e_ == cudaErrorMemoryAllocation ? FMMLU_ERR_OOM : FMMLU_ERR_CUDA,        \
                  std::string(#x) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

constexpr uint32_t kTreeMagic = 0x54554d46u;    // "FMUT"
constexpr uint32_t kHandleMagic = 0x48554d46u;  // "FMUH"

// Host-side time of a factorization (stats "host_ms"): device allocation and
// release, waits for the stream, level set-up; accumulated on the thread
// that runs the factorization.
struct HostTimes {
  double alloc = 0, release = 0, wait = 0, make_level = 0, plan = 0, setup = 0;
  double setup_desc = 0, setup_pairs = 0, setup_plans = 0;
  int64_t allocs = 0;
};
thread_local HostTimes* g_ht = nullptr;

struct HostTimer {
  double* acc;
  std::chrono::steady_clock::time_point t0;
  explicit HostTimer(double HostTimes::*m)
      : acc(g_ht ? &(g_ht->*m) : nullptr), t0(std::chrono::steady_clock::now()) {}
  ~HostTimer() {
    if (acc)
      *acc += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                  .count();
  }
};

inline void stream_wait(cudaStream_t st) {
  HostTimer t(&HostTimes::wait);
  CK(cudaStreamSynchronize(st));
}

template <typename T>
T* dalloc(size_t count) {
  if (count == 0) count = 1;
  void* p = nullptr;
  HostTimer t(&HostTimes::alloc);
  if (g_ht) ++g_ht->allocs;
  CK(cudaMalloc(&p, count * sizeof(T)));
  return static_cast<T*>(p);
}

template <typename T>
T* dupload(const std::vector<T>& v, cudaStream_t st) {
  T* p = dalloc<T>(v.size());
  if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return p;
}

template <typename T>
std::vector<T> ddownload(const T* p, size_t count, cudaStream_t st) {
  std::vector<T> v(count);
  if (count) CK(cudaMemcpyAsync(v.data(), p, count * sizeof(T), cudaMemcpyDeviceToHost, st));
  stream_wait(st);
  return v;
}

// owns device allocations, freed in reverse order
struct DevPool {
  std::vector<void*> ptrs;
  template <typename T>
  T* get(size_t count) {
    T* p = dalloc<T>(count);
    ptrs.push_back(p);
    return p;
  }
  template <typename T>
  T* up(const std::vector<T>& v, cudaStream_t st) {
    T* p = dupload(v, st);
    ptrs.push_back(p);
    return p;
  }
  void release() {
    HostTimer t(&HostTimes::release);
    for (auto it = ptrs.rbegin(); it != ptrs.rend(); ++it) cudaFree(*it);
    ptrs.clear();
  }
  ~DevPool() { release(); }
};

// Scratch buffers reused from one level to the next: the k-th request of a
// level gets the k-th slot, grown (freed and allocated larger) only when it
// is too small, so a factorization allocates each scratch buffer a few times
// instead of once per level. Uploads are stream-ordered after the work that
// read the slot's previous contents; growing frees through cudaFree, which
// waits for the device.
struct ScratchPool {
  std::vector<std::pair<void*, size_t>> slots;
  size_t next = 0;
  void reset() { next = 0; }
  template <typename T>
  T* get(size_t count) {
    const size_t bytes = std::max<size_t>(1, count) * sizeof(T);
    if (next == slots.size()) slots.push_back({nullptr, 0});
    auto& sl = slots[next++];
    if (sl.second < bytes) {
      if (sl.first) {
        HostTimer t(&HostTimes::release);
        cudaFree(sl.first);
      }
      sl.first = nullptr;
      sl.second = 0;
      sl.first = dalloc<unsigned char>(bytes);
      sl.second = bytes;
    }
    return static_cast<T*>(sl.first);
  }
  template <typename T>
  T* up(const std::vector<T>& v, cudaStream_t st) {
    T* p = get<T>(v.size());
    if (!v.empty())
      CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return p;
  }
  ~ScratchPool() {
    for (auto& sl : slots)
      if (sl.first) cudaFree(sl.first);
  }
};

// Device buffers in numbered slots, grown (never shrunk) on demand: the
// Schur pools of the levels alternate between two slots, so a factorization
// allocates a pool only when a level needs more than its slot holds and
// frees them all at its end (a cudaFree waits for the device).
struct DevSlots {
  std::vector<std::pair<void*, size_t>> slots;
  template <typename T>
  T* get(int slot, size_t count) {
    if ((int)slots.size() <= slot) slots.resize((size_t)slot + 1, {nullptr, 0});
    auto& sl = slots[(size_t)slot];
    const size_t bytes = std::max<size_t>(1, count) * sizeof(T);
    if (sl.second < bytes) {
      if (sl.first) {
        HostTimer t(&HostTimes::release);
        cudaFree(sl.first);
      }
      sl.first = nullptr;
      sl.second = 0;
      sl.first = dalloc<unsigned char>(bytes);
      sl.second = bytes;
    }
    return static_cast<T*>(sl.first);
  }
  ~DevSlots() {
    for (auto& sl : slots)
      if (sl.first) cudaFree(sl.first);
  }
};

// Pinned host buffers in numbered slots, grown (never shrunk) on demand.
struct PinnedPool {
  std::vector<std::pair<void*, size_t>> slots;
  template <typename T>
  T* get(int slot, size_t count) {
    if ((int)slots.size() <= slot) slots.resize((size_t)slot + 1, {nullptr, 0});
    auto& sl = slots[(size_t)slot];
    const size_t bytes = std::max<size_t>(1, count) * sizeof(T);
    if (sl.second < bytes) {
      if (sl.first) cudaFreeHost(sl.first);
      sl.first = nullptr;
      sl.second = 0;
      CK(cudaMallocHost(&sl.first, bytes));
      sl.second = bytes;
    }
    return static_cast<T*>(sl.first);
  }
  ~PinnedPool() {
    for (auto& sl : slots)
      if (sl.first) cudaFreeHost(sl.first);
  }
};


// A unit list of tcgen05 launches: pinned host staging and its device copy.
// The staging buffer is rewritten only after the previous copy out of it has
// run (event); the device copy is stream-ordered after the launches that read
// the previous list. Growing waits for the stream (the old buffers may still
// be read).
struct UnitBuf {
  TcUnit* h = nullptr;
  TcUnit* d = nullptr;
  size_t cap = 0;
  cudaEvent_t copied = nullptr;
  bool pending = false;
  void upload(const std::vector<TcUnit>& u, cudaStream_t st) {
    if (u.empty()) return;
    if (!copied) CK(cudaEventCreateWithFlags(&copied, cudaEventDisableTiming));
    if (pending) {
      HostTimer t(&HostTimes::wait);
      CK(cudaEventSynchronize(copied));
    }
    pending = false;
    if (u.size() > cap) {
      stream_wait(st);
      release_buffers();
      cap = std::max(u.size(), (size_t)4096);
      CK(cudaMallocHost(&h, cap * sizeof(TcUnit)));
      CK(cudaMalloc(&d, cap * sizeof(TcUnit)));
    }
    std::memcpy(h, u.data(), u.size() * sizeof(TcUnit));
    CK(cudaMemcpyAsync(d, h, u.size() * sizeof(TcUnit), cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(copied, st));
    pending = true;
  }
  void release_buffers() {
    if (h) cudaFreeHost(h);
    if (d) cudaFree(d);
    h = nullptr;
    d = nullptr;
    cap = 0;
  }
  ~UnitBuf() {
    if (pending) cudaEventSynchronize(copied);
    release_buffers();
    if (copied) cudaEventDestroy(copied);
  }
};

constexpr int kRowChunkHost = 16;   // rows per CTA of the solve's R and S products
// Real flops of one ID-matrix entry: comb_kernel_pair evaluates an entry and
// its transpose partner from one distance in 51 adds and multiplies (the
// coordinate differences, r^2, sqrt, 1/r^2, G, G (ikr - 1), both normal
// projections, both combined-field values, the sqrt(w) scaling) plus one
// sincos, which is not counted.
constexpr double kKevalFlops = 25.5;

inline uint64_t pkey(int x, int y) { return ((uint64_t)(uint32_t)x << 32) | (uint32_t)y; }

void default_opts(fmmlu_opts* o) {
  o->leaf_size = 64;
  o->eta = NAN;
  o->proxy_radius_factor = 1.5;
  o->n_proxy = 300;
  o->proxy_rule = FMMLU_PROXY_FIXED;
  o->precision = FMMLU_PRECISION_AUTO;
  o->eps_id_divisor = 1.0;
  o->verbose = 0;
  o->profile = 0;
  o->cpqr_single = 0;
  o->schur_emulation = 1;
  o->id_method = FMMLU_ID_AUTO;
  o->xrr_refine_tol = 1e-9;
  o->solve_chunk = 0;
  o->solve_graph = 1;
  o->solve_tc_nrhs = 32;
  o->autotune = 1;
  o->autotune_cache = nullptr;
}

fmmlu_opts checked_opts(const fmmlu_opts* in) {
  fmmlu_opts o;
  default_opts(&o);
  if (in) o = *in;
  if (o.leaf_size < 1 || o.leaf_size > 4096) throw Error(FMMLU_ERR_INVALID_ARG, "leaf_size out of [1, 4096]");
  if (!(o.proxy_radius_factor > 1.0 && o.proxy_radius_factor < 2.88))
    throw Error(FMMLU_ERR_INVALID_ARG, "proxy_radius_factor must lie in (1, 2.88)");
  if (o.n_proxy < 8 || o.n_proxy > 100000) throw Error(FMMLU_ERR_INVALID_ARG, "n_proxy out of [8, 100000]");
  if (o.proxy_rule != FMMLU_PROXY_FIXED && o.proxy_rule != FMMLU_PROXY_ADAPTIVE)
    throw Error(FMMLU_ERR_INVALID_ARG, "proxy_rule must be FMMLU_PROXY_FIXED or FMMLU_PROXY_ADAPTIVE");
  if (o.precision < 0 || o.precision > 2) throw Error(FMMLU_ERR_INVALID_ARG, "bad precision");
  if (!(o.eps_id_divisor > 0.0)) throw Error(FMMLU_ERR_INVALID_ARG, "eps_id_divisor must be > 0");
  if (o.id_method < 0 || o.id_method > 2) throw Error(FMMLU_ERR_INVALID_ARG, "bad id_method");
  if (o.schur_emulation < 0 || o.schur_emulation > 2) throw Error(FMMLU_ERR_INVALID_ARG, "bad schur_emulation");
  if (std::isnan(o.xrr_refine_tol)) throw Error(FMMLU_ERR_INVALID_ARG, "xrr_refine_tol is NaN");
  if (o.solve_chunk != 0 && (o.solve_chunk < 16 || o.solve_chunk > 4096 || o.solve_chunk % 16))
    throw Error(FMMLU_ERR_INVALID_ARG, "solve_chunk must be 0 or a multiple of 16 in [16, 4096]");
  if (o.solve_graph < 0 || o.solve_graph > 2) throw Error(FMMLU_ERR_INVALID_ARG, "bad solve_graph");
  if (o.solve_tc_nrhs < 0) throw Error(FMMLU_ERR_INVALID_ARG, "solve_tc_nrhs must be >= 0");
  if (o.autotune < 0 || o.autotune > 1) throw Error(FMMLU_ERR_INVALID_ARG, "bad autotune");
  return o;
}

}  // namespace

struct fmmlu_tree {
  uint32_t magic = kTreeMagic;
  TreeHost T;
  int* d_perm = nullptr;
  fmmlu_opts opts;
  ~fmmlu_tree() { if (d_perm) cudaFree(d_perm); }
};

namespace {

// The chunk items of the solve sweeps for one chunk size (rows of C per CTA
// in the forward sweep, columns in the backward one), on the device.
// Launch lists of the C products of the sweeps on the tensor cores for one
// (nrhs, direction): per colour the unit lists of the operand splits and the
// product tiles, and per box the offsets of its digit slices and exponents in
// a per-colour scratch (the C and T products of a colour reuse it in turn).
struct TcSolvePlan {
  DevPool mem;
  TcUnit* d_units = nullptr;
  TcBoxHost* d_tbC = nullptr;
  TcBoxHost* d_tbT = nullptr;
  std::vector<TcPlan> plC, plT;   // per colour segment
  int64_t slice_bytes = 256, expo_ints = 64;
};

struct SolvePlan {
  int chunk = 0;
  DevPool mem;
  SolveBox* d_boxes = nullptr;
  SweepItem* d_items = nullptr;
  std::vector<SweepSeg> segs;   // elimination order
  int64_t part_max = 1;         // partial sums per right-hand side (backward sweep)
  // tensor-core products: placeholder descriptors (one per box, zero) and a
  // status word for the generic product kernels, and the launch lists
  BoxDesc* d_desc = nullptr;
  BoxRun* d_run = nullptr;
  int* d_status = nullptr;
  std::map<std::pair<int, int>, std::shared_ptr<TcSolvePlan>> tc;   // (nrhs, adjoint)
};

// Work vectors of the solves with one (nrhs, direction, stream, chunk) and,
// once that key has been used before (or always, by option), the sweeps
// captured as one CUDA graph that later solves replay.
struct SolveCtx {
  int nrhs = 0;
  bool adjoint = false;
  cudaStream_t stream = nullptr;
  std::shared_ptr<SolvePlan> plan;
  DevPool mem;
  double2 *v = nullptr, *part = nullptr, *vr = nullptr, *z = nullptr;
  int* cnt = nullptr;           // per box and right-hand side: backward chunks done
  void* rscr = nullptr;
  std::shared_ptr<TcSolvePlan> tcp;   // C products on the tensor cores (else fp64)
  unsigned char* tslices = nullptr;
  int* texpo = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_kernels = 0;
  int64_t uses = 0;
  uint64_t last = 0;
  cudaEvent_t done = nullptr;   // recorded after each use on `stream`
  ~SolveCtx() {
    if (done) {
      cudaEventSynchronize(done);
      cudaEventDestroy(done);
    }
    if (exec) cudaGraphExecDestroy(exec);
  }
};

}  // namespace

struct fmmlu_handle {
  uint32_t magic = kHandleMagic;
  int device = -1;             // CUDA device current at fmmlu_factor (holds the factors)
  int64_t n = 0;
  double k = 0, eta = 0, eps = 0;
  bool fp32 = false;
  bool gram = false;           // ID by pivoted Cholesky of M^H M
  DevPool mem;                 // factors, plans, permutation
  int* d_perm = nullptr;
  std::vector<SolveBox> sboxes;   // eliminated boxes in elimination order (host)
  std::vector<SweepSeg> sseg;     // their colour segments (items not yet built)
  int chunk0 = kSweepChunkDefault;
  int solve_graph = 1, autotune = 0;
  int solve_tc_nrhs = 32;         // tensor-core C products from this many rhs (0: never)
  std::string tune_cache;
  uint64_t shape_key = 0;         // hash of the solve structure (tuning cache key)
  int n0 = 0, nb_root = 64;
  int* d_root_dofs = nullptr;
  double2* d_root = nullptr;
  std::string stats;
  int64_t factor_entries = 0;  // complex entries of the stored factors (m_f / 16)
  int64_t arena_bytes = 0;
  bool profile = false;
  mutable Profiler prof;       // per-kernel accounting (factor + solves)
  mutable std::mutex smu;      // guards the solve state below
  mutable std::map<int, std::shared_ptr<SolvePlan>> plans;   // by chunk
  mutable std::map<std::pair<int, int>, int> chunk_for;      // (nrhs, adjoint) -> chunk
  mutable std::vector<std::unique_ptr<SolveCtx>> ctxs;
  mutable cudaStream_t cap_stream = nullptr;
  mutable uint64_t tick = 0;
  ~fmmlu_handle() {
    ctxs.clear();
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

namespace {

// ---------------------------------------------------------------------------
// level state
// ---------------------------------------------------------------------------

// tree id -> current index (-1: not current), a flat table over all boxes
struct CurIndex {
  std::vector<int> v;
  void reset(size_t nboxes) { v.assign(nboxes, -1); }
  int find(int id) const { return id >= 0 && (size_t)id < v.size() ? v[id] : -1; }
  int at(int id) const {
    const int c = find(id);
    if (c < 0) throw Error(FMMLU_ERR_CUDA, "internal: box not current");
    return c;
  }
};

// Run f(begin, end) over [0, n) on up to 16 host threads (contiguous
// ranges, so per-range results concatenate in order). f must not throw.
template <class F>
void parallel_for(int64_t n, F f) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int64_t nt = std::min<int64_t>(std::min<unsigned>(16u, hw), std::max<int64_t>(1, n / 2048));
  if (nt <= 1) {
    f((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  const int64_t chunk = (n + nt - 1) / nt;
  for (int64_t t = 0; t < nt; ++t) {
    const int64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b < e) th.emplace_back([=, &f] { f(b, e); });
  }
  for (auto& x : th) x.join();
}

// The Schur blocks of one level: for every current box x the sorted list of
// the boxes y that have a block (x, y) with x's rows, and each block's offset
// in the pool (blocks are laid out x-major, then by y).
struct PairCSR {
  std::vector<int64_t> start;   // nc + 1
  std::vector<int> ys;
  std::vector<int64_t> off;
  int64_t find(int x, int y) const {
    if (x < 0 || (size_t)x + 1 >= start.size()) return -1;
    const int* b = ys.data() + start[x];
    const int* e = ys.data() + start[x + 1];
    const int* it = std::lower_bound(b, e, y);
    return (it != e && *it == y) ? off[it - ys.data()] : -1;
  }
  int64_t at(int x, int y) const {
    const int64_t v = find(x, y);
    if (v < 0) throw Error(FMMLU_ERR_CUDA, "internal: missing Schur pair");
    return v;
  }
  size_t size() const { return ys.size(); }
};

struct LevelState {
  int level = 0;
  std::vector<int> cur;                    // tree ids of current boxes
  CurIndex cidx;                           // tree id -> current index
  std::vector<int> a0, off;                // per current box
  std::vector<int> act_dof;                // level-start DOFs (concatenated)
  std::vector<int> cur_n, act_pos;         // after processing (host copies)
  PairCSR pair;                            // (cur x, cur y) -> pool offset
  DevPool mem;
  int *d_cur_n = nullptr, *d_cur_off = nullptr, *d_cur_a0 = nullptr;
  int *d_act_dof = nullptr, *d_act_pos = nullptr;
  double2* d_pool = nullptr;
  int64_t pool_size = 0;
  int64_t total() const { return (int64_t)act_dof.size(); }
  // current active DOFs of current box c (after processing)
  void active_dofs(int c, std::vector<int>& out) const {
    for (int i = 0; i < cur_n[c]; ++i) out.push_back(act_dof[off[c] + act_pos[off[c] + i]]);
  }
};

std::unique_ptr<LevelState> make_level(const TreeHost& T, int level, const LevelState* prev,
                                       const HLevel* lists, cudaStream_t st, DevSlots* pools) {
  auto L = std::make_unique<LevelState>();
  L->level = level;
  L->cur = current_boxes(T, level);
  int nc = (int)L->cur.size();
  L->cidx.reset(T.boxes.size());
  for (int c = 0; c < nc; ++c) L->cidx.v[L->cur[c]] = c;
  L->a0.resize(nc);
  L->off.resize(nc);
  for (int c = 0; c < nc; ++c) {
    int X = L->cur[c];
    const HBox& b = T.boxes[X];
    L->off[c] = (int)L->act_dof.size();
    if (b.level == level && !b.leaf()) {
      for (int ch : b.kids) {
        prev->active_dofs(prev->cidx.at(ch), L->act_dof);
      }
    } else {
      for (int64_t p = b.start; p < b.end; ++p) L->act_dof.push_back((int)p);
    }
    L->a0[c] = (int)L->act_dof.size() - L->off[c];
  }
  L->cur_n = L->a0;
  L->act_pos.resize(L->act_dof.size());
  for (int c = 0; c < nc; ++c)
    for (int i = 0; i < L->a0[c]; ++i) L->act_pos[L->off[c] + i] = i;
  // pair set: images of the previous pairs, plus closed-neighbourhood pairs.
  // Built per row box x without hashing: the candidate columns of x are the
  // images of the previous pairs whose row maps to x and the closed
  // neighbourhoods {B} u N(B) that contain x; a per-thread stamp array drops
  // duplicates, and every row is sorted.
  std::vector<int> img;   // previous current box -> its image at this level
  if (prev) {
    img.resize(prev->cur.size());
    for (size_t c = 0; c < prev->cur.size(); ++c) {
      const HBox& b = T.boxes[prev->cur[c]];
      img[c] = L->cidx.at(b.level == level + 1 ? b.parent : prev->cur[c]);
    }
  }
  // previous pairs grouped by the image of their row: rows of prev map to x
  std::vector<int64_t> pstart(nc + 1, 0);
  std::vector<int> prow_src;   // previous rows, grouped by image
  if (prev) {
    for (size_t c = 0; c < prev->cur.size(); ++c) ++pstart[img[c] + 1];
    for (int c = 0; c < nc; ++c) pstart[c + 1] += pstart[c];
    prow_src.resize(prev->cur.size());
    std::vector<int64_t> fill(pstart.begin(), pstart.end() - 1);
    for (size_t c = 0; c < prev->cur.size(); ++c) prow_src[fill[img[c]]++] = (int)c;
  }
  // closed neighbourhoods, and for every x the level boxes whose
  // neighbourhood holds it
  std::vector<int64_t> cnb;   // per level box: start into cn
  std::vector<int> cn;
  std::vector<int64_t> istart(nc + 1, 0);
  std::vector<int> inv;
  if (lists) {
    const size_t nbx = lists->boxes.size();
    cnb.resize(nbx + 1, 0);
    for (size_t r = 0; r < nbx; ++r) {
      cnb[r] = (int64_t)cn.size();
      cn.push_back(L->cidx.at(lists->boxes[r]));
      for (int j = lists->nbeg[r]; j < lists->nbeg[r] + lists->ncnt[r]; ++j)
        cn.push_back(L->cidx.at(lists->nlist[j]));
    }
    cnb[nbx] = (int64_t)cn.size();
    for (int x : cn) ++istart[x + 1];
    for (int c = 0; c < nc; ++c) istart[c + 1] += istart[c];
    inv.resize(cn.size());
    std::vector<int64_t> fill(istart.begin(), istart.end() - 1);
    for (size_t r = 0; r < nbx; ++r)
      for (int64_t q = cnb[r]; q < cnb[r + 1]; ++q) inv[fill[cn[q]]++] = (int)r;
  }
  // rows, in parallel over contiguous ranges of x
  std::vector<int64_t> rcount(nc, 0);
  std::vector<std::vector<int>> parts;
  std::mutex pmu;
  std::vector<std::pair<int64_t, int>> part_of;   // range begin -> part index
  parallel_for(nc, [&](int64_t x0, int64_t x1) {
    std::vector<int> stamp(nc, -1), row, out;
    for (int64_t x = x0; x < x1; ++x) {
      row.clear();
      auto take = [&](int y) {
        if (stamp[y] != (int)x) { stamp[y] = (int)x; row.push_back(y); }
      };
      if (prev)
        for (int64_t q = pstart[x]; q < pstart[x + 1]; ++q) {
          const int xp = prow_src[q];
          const PairCSR& P = prev->pair;
          for (int64_t e = P.start[xp]; e < P.start[xp + 1]; ++e) take(img[P.ys[e]]);
        }
      for (int64_t q = istart[x]; q < istart[x + 1]; ++q) {
        const int r = inv[q];
        for (int64_t e = cnb[r]; e < cnb[r + 1]; ++e) take(cn[e]);
      }
      std::sort(row.begin(), row.end());
      rcount[x] = (int64_t)row.size();
      out.insert(out.end(), row.begin(), row.end());
    }
    std::lock_guard<std::mutex> lk(pmu);
    part_of.push_back({x0, (int)parts.size()});
    parts.push_back(std::move(out));
  });
  std::sort(part_of.begin(), part_of.end());
  PairCSR& P = L->pair;
  P.start.assign(nc + 1, 0);
  for (int x = 0; x < nc; ++x) P.start[x + 1] = P.start[x] + rcount[x];
  P.ys.reserve((size_t)P.start[nc]);
  for (auto& po : part_of) P.ys.insert(P.ys.end(), parts[po.second].begin(), parts[po.second].end());
  parts.clear();
  P.off.resize(P.ys.size());
  int64_t tot = 0;
  for (int x = 0; x < nc; ++x)
    for (int64_t e = P.start[x]; e < P.start[x + 1]; ++e) {
      P.off[e] = tot;
      tot += (int64_t)L->a0[x] * L->a0[P.ys[e]];
    }
  L->pool_size = tot;
  L->d_pool = pools ? pools->get<double2>(level & 1, (size_t)tot) : L->mem.get<double2>((size_t)tot);
  if (tot) CK(cudaMemsetAsync(L->d_pool, 0, (size_t)tot * sizeof(double2), st));
  L->d_cur_n = L->mem.up(L->cur_n, st);
  L->d_cur_off = L->mem.up(L->off, st);
  L->d_cur_a0 = L->mem.up(L->a0, st);
  L->d_act_dof = L->mem.up(L->act_dof, st);
  L->d_act_pos = L->mem.up(L->act_pos, st);
  // gather the previous Schur blocks into the new pool
  if (prev && prev->pair.size() > 0) {
    std::vector<int> suboff(prev->cur.size(), 0);   // offset of prev box inside its image
    {
      std::vector<int> run(nc, 0);   // image -> running offset (children in order)
      for (size_t c = 0; c < prev->cur.size(); ++c) {
        const HBox& b = T.boxes[prev->cur[c]];
        if (b.level == level + 1) {
          // children of one parent are consecutive in current order (by start)
          int& o = run[img[c]];
          suboff[c] = o;
          o += prev->cur_n[c];
        }
      }
    }
    const PairCSR& Q = prev->pair;
    const int npc = (int)prev->cur.size();
    std::vector<std::vector<MergeItem>> iparts;
    std::vector<std::pair<int64_t, int>> ipart_of;
    bool missing = false;
    parallel_for(npc, [&](int64_t x0, int64_t x1) {
      std::vector<MergeItem> items;
      bool miss = false;
      for (int64_t x = x0; x < x1; ++x)
        for (int64_t e = Q.start[x]; e < Q.start[x + 1]; ++e) {
          const int y = Q.ys[e];
          const int X = img[x], Y = img[y];
          MergeItem it;
          const int64_t dst = L->pair.find(X, Y);
          if (dst < 0) { miss = true; continue; }
          it.src = prev->d_pool + Q.off[e];
          it.dst = L->d_pool + dst;
          it.ld_src = prev->a0[x];
          it.ld_dst = L->a0[X];
          it.off_i = suboff[x];
          it.off_j = suboff[y];
          it.ni = prev->cur_n[x];
          it.nj = prev->cur_n[y];
          it.pos_i = prev->d_act_pos + prev->off[x];
          it.pos_j = prev->d_act_pos + prev->off[y];
          if (it.ni > 0 && it.nj > 0) items.push_back(it);
        }
      std::lock_guard<std::mutex> lk(pmu);
      missing = missing || miss;
      ipart_of.push_back({x0, (int)iparts.size()});
      iparts.push_back(std::move(items));
    });
    if (missing) throw Error(FMMLU_ERR_CUDA, "internal: missing Schur pair");
    std::sort(ipart_of.begin(), ipart_of.end());
    std::vector<MergeItem> items;
    for (auto& po : ipart_of) items.insert(items.end(), iparts[po.second].begin(), iparts[po.second].end());
    MergeItem* d_items = L->mem.up(items, st);
    launch_merge(d_items, (int)items.size(), 0, 0, st);
    CK(cudaGetLastError());
  }
  return L;
}

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

int status_to_code(int s, std::string& msg) {
  if (s & kStatusSingular) { msg = "singular pivot in X_RR or a root block"; return FMMLU_ERR_SINGULAR_PIVOT; }
  if (s & kStatusNonfinite) { msg = "non-finite value in an ID matrix"; return FMMLU_ERR_NONFINITE; }
  if (s & kStatusBound) { msg = "internal size bound exceeded"; return FMMLU_ERR_LIMIT; }
  if (s & kStatusTimeout) { msg = "a bounded inter-CTA wait gave up"; return FMMLU_ERR_TIMEOUT; }
  return 0;
}

// process-wide tuning results (key -> chunk), optionally kept in text files
// of "key value" lines: a file is read on first use and every result this
// process uses that the file lacks is appended to it
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
std::map<std::string, std::set<std::string>> g_tune_files;

bool valid_chunk(int c) { return c >= 16 && c <= 4096 && c % 16 == 0; }

std::set<std::string>& tune_file_keys(const std::string& path) {
  auto it = g_tune_files.find(path);
  if (it != g_tune_files.end()) return it->second;
  std::set<std::string>& keys = g_tune_files[path];
  std::ifstream f(path);
  std::string k;
  long v;
  while (f >> k >> v)
    if (valid_chunk((int)v)) {
      g_tune[k] = (int)v;
      keys.insert(k);
    }
  return keys;
}

bool tune_lookup(const std::string& path, const std::string& key, int* out) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (!path.empty()) tune_file_keys(path);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}

void tune_store(const std::string& path, const std::string& key, int v) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = v;
  if (path.empty()) return;
  std::set<std::string>& keys = tune_file_keys(path);
  if (keys.count(key)) return;
  std::ofstream f(path, std::ios::app);
  if (f) {
    f << key << ' ' << v << '\n';
    keys.insert(key);
  }
}

std::string device_tag() {
  int dev = 0;
  cudaDeviceProp pr{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&pr, dev) != cudaSuccess)
    return "unknown";
  std::string s = pr.name;
  for (char& ch : s)
    if (ch == ' ' || ch == '\t' || ch == '\n') ch = '_';
  return s + "_sm" + std::to_string(pr.major) + std::to_string(pr.minor);
}

// k16 steps per split-K chunk of a colour's Gram product. With autotune on,
// the colour's shape (log2 buckets of its upper-triangle tiles and of its
// longest k range) is looked up in the process-wide tuning results; on a
// miss every candidate runs once on this colour (all give the same exact
// sums) and the fastest is kept.
template <class Run>
int gram_chunk_for(const fmmlu_opts& opt, const std::vector<TcBoxSize>& bs, bool fp32,
                   cudaStream_t st, Run&& run) {
  if (!opt.autotune) return kGramChunkDefault;
  int64_t tiles = 0, ks = 1;
  for (const TcBoxSize& b : bs) {
    const int64_t t = (b.a + 127) / 128, tn = (b.a + 31) / 32;
    tiles += t * tn;
    ks = std::max<int64_t>(ks, (b.kgram + 15) / 16);
  }
  auto lg = [](int64_t v) { int l = 0; while (v > 1) { v >>= 1; ++l; } return l; };
  const std::string key = "gram_chunk|" + device_tag() + "|" + (fp32 ? "c64" : "c128") +
                          "|tiles=" + std::to_string(lg(tiles)) + "|ks=" + std::to_string(lg(ks));
  const std::string path = opt.autotune_cache ? opt.autotune_cache : "";
  int chunk = 0;
  if (!tune_lookup(path, key, &chunk)) {
    ProfScope none(nullptr);
    struct Ev {
      cudaEvent_t e = nullptr;
      ~Ev() { if (e) cudaEventDestroy(e); }
    } e0, e1;
    CK(cudaEventCreate(&e0.e));
    CK(cudaEventCreate(&e1.e));
    float best = INFINITY;
    chunk = kGramChunkDefault;
    for (int c : {32, 64, 128, 256, 4096}) {
      CK(cudaEventRecord(e0.e, st));
      run(c);
      CK(cudaEventRecord(e1.e, st));
      CK(cudaEventSynchronize(e1.e));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0.e, e1.e));
      if (ms < best) {
        best = ms;
        chunk = c;
      }
    }
  }
  tune_store(path, key, chunk);
  return chunk;
}

// Chunk items of the solve sweeps for one chunk size: per box, C = [S | N]
// in chunks of `chunk` rows (each chunk owns r partial sums, which the first
// chunk also uses as the box's z scratch), and R and S in chunks of
// kRowChunkHost rows.
std::shared_ptr<SolvePlan> make_solve_plan(const fmmlu_handle* H, int chunk, cudaStream_t st) {
  auto P = std::make_shared<SolvePlan>();
  P->chunk = chunk;
  std::vector<SolveBox> boxes = H->sboxes;
  std::vector<SweepItem> items;
  P->segs = H->sseg;
  for (SweepSeg& sg : P->segs) {
    int64_t part = 0;
    sg.chunk = chunk;
    sg.i0 = (int)items.size();
    for (int q = sg.b0; q < sg.b0 + sg.nb; ++q) {
      SolveBox& sb = boxes[q];
      sb.zoff = (int)part;
      sb.item_beg = (int)items.size();
      const int c = sb.s + sb.n;
      for (int c0 = 0; c0 == 0 || c0 < c; c0 += chunk) {
        items.push_back(SweepItem{q, c0, std::min(c, c0 + chunk), (int)part});
        part += sb.r;
      }
      sb.item_cnt = (int)items.size() - sb.item_beg;
      sb.toff = (int)part;
      part += sb.r;
    }
    sg.ni = (int)items.size() - sg.i0;
    sg.ri0 = (int)items.size();
    for (int q = sg.b0; q < sg.b0 + sg.nb; ++q)
      for (int k0 = 0; k0 < boxes[q].r; k0 += kRowChunkHost)
        items.push_back(SweepItem{q, k0, std::min(boxes[q].r, k0 + kRowChunkHost), 0});
    sg.nri = (int)items.size() - sg.ri0;
    sg.si0 = (int)items.size();
    for (int q = sg.b0; q < sg.b0 + sg.nb; ++q)
      for (int i0 = 0; i0 < boxes[q].s; i0 += kRowChunkHost)
        items.push_back(SweepItem{q, i0, std::min(boxes[q].s, i0 + kRowChunkHost), 0});
    sg.nsi = (int)items.size() - sg.si0;
    sg.part = part;
    P->part_max = std::max(P->part_max, part);
  }
  if (items.size() > (size_t)INT32_MAX) throw Error(FMMLU_ERR_LIMIT, "too many solve items");
  P->d_boxes = P->mem.up(boxes, st);
  P->d_items = P->mem.up(items, st);
  const size_t nbx = std::max<size_t>(1, boxes.size());
  P->d_desc = P->mem.get<BoxDesc>(nbx);
  P->d_run = P->mem.get<BoxRun>(nbx);
  P->d_status = P->mem.get<int>(1);
  CK(cudaMemsetAsync(P->d_desc, 0, nbx * sizeof(BoxDesc), st));
  CK(cudaMemsetAsync(P->d_run, 0, nbx * sizeof(BoxRun), st));
  CK(cudaMemsetAsync(P->d_status, 0, sizeof(int), st));
  return P;
}

// Launch lists of the tensor-core C products of plan P for nrhs right-hand
// sides in one direction (the adjoint products read the other block,
// transposed, which changes how their exponent passes are laid out).
std::shared_ptr<TcSolvePlan> get_tc_solve_plan(const fmmlu_handle* H, SolvePlan& P, int nrhs,
                                               bool adjoint, cudaStream_t st) {
  const auto key = std::make_pair(nrhs, adjoint ? 1 : 0);
  auto it = P.tc.find(key);
  if (it != P.tc.end()) return it->second;
  auto tp = std::make_shared<TcSolvePlan>();
  const size_t nbx = H->sboxes.size();
  std::vector<TcBoxHost> tbC(std::max<size_t>(1, nbx)), tbT(std::max<size_t>(1, nbx));
  std::vector<TcUnit> units;
  for (const SweepSeg& sg : P.segs) {
    std::vector<TcBoxSize> bs(sg.nb);
    int64_t so = 0, eo = 0, so2 = 0, eo2 = 0;
    for (int q = 0; q < sg.nb; ++q) {
      const SolveBox& sb = H->sboxes[sg.b0 + q];
      bs[q] = TcBoxSize{0, sb.s, sb.r, sb.n, 0, 0, nrhs};
      plan_tc_box(sb.s + sb.n, nrhs, sb.r, 7, so, eo, tbC[sg.b0 + q]);
      plan_tc_box(sb.r, nrhs, sb.s + sb.n, 7, so2, eo2, tbT[sg.b0 + q]);
    }
    tp->slice_bytes = std::max(tp->slice_bytes, std::max(so, so2));
    tp->expo_ints = std::max(tp->expo_ints, std::max(eo, eo2));
    TcPlan pc{}, pt{};
    tc_plan(adjoint ? kTcSvCA : kTcSvC, bs, units, pc);
    tc_plan(adjoint ? kTcSvTA : kTcSvT, bs, units, pt);
    tp->plC.push_back(pc);
    tp->plT.push_back(pt);
  }
  if (units.empty()) units.push_back(TcUnit{0, 0, 0, 0});
  tp->d_units = tp->mem.up(units, st);
  tp->d_tbC = tp->mem.up(tbC, st);
  tp->d_tbT = tp->mem.up(tbT, st);
  P.tc[key] = tp;
  return tp;
}

// Proxy points per sphere of radius rho (Sec. 5.2: n_gamma from multipole
// estimates). Adaptive rule: the excess-bandwidth truncation degree
// p = ceil(k rho + 1.8 d^(2/3) (k rho)^(1/3)), d = log10(1/eps), and
// 2 (p + 1)^2 points (twice the spherical harmonics of degree <= p), at least
// n_proxy.
int proxy_count_for(const fmmlu_opts& opt, double k, double rho, double eps) {
  if (opt.proxy_rule != FMMLU_PROXY_ADAPTIVE) return opt.n_proxy;
  const double kr = k * rho, d0 = std::log10(1.0 / eps);
  const double p = std::ceil(kr + 1.8 * std::pow(d0, 2.0 / 3.0) * std::pow(kr, 1.0 / 3.0));
  const double cnt = 2.0 * (p + 1.0) * (p + 1.0);
  if (!(cnt < 1e6)) throw Error(FMMLU_ERR_LIMIT, "adaptive proxy count above 10^6 points");
  return std::max(opt.n_proxy, (int)cnt);
}

void factor_impl(const fmmlu_tree* tree, const double* pts, const double* nrm, const double* w,
                 double k, double eps, const fmmlu_opts& opt, cudaStream_t st, fmmlu_handle* H) {
  const TreeHost& T = tree->T;
  const int64_t n = T.n;
  CK(cudaGetDevice(&H->device));
  H->n = n;
  H->k = k;
  H->eta = std::isnan(opt.eta) ? k : opt.eta;
  H->eps = eps;
  H->fp32 = opt.precision == FMMLU_PRECISION_MIXED ||
            (opt.precision == FMMLU_PRECISION_AUTO && eps >= 1e-5);
  const double eps_id = eps / opt.eps_id_divisor;
  // Gram form of the ID: fp64 rounding of G = M^H M is ~1e-16 |G|, far below
  // the eps_ID^2 |G| the rank rule must resolve while eps_ID >= 1e-7
  const bool use_gram = opt.id_method == FMMLU_ID_GRAM ||
                        (opt.id_method == FMMLU_ID_AUTO && eps_id >= 1e-7);
  H->gram = use_gram;
  H->profile = opt.profile != 0;
  H->chunk0 = opt.solve_chunk > 0 ? opt.solve_chunk : kSweepChunkDefault;
  H->solve_graph = opt.solve_graph;
  H->solve_tc_nrhs = opt.solve_tc_nrhs;
  H->autotune = opt.solve_chunk == 0 ? opt.autotune : 0;
  H->tune_cache = opt.autotune_cache ? opt.autotune_cache : "";
  ProfScope prof_scope(H->profile ? &H->prof : nullptr);
  HostTimes ht;
  struct HtScope {
    HostTimes* saved;
    explicit HtScope(HostTimes* p) : saved(g_ht) { g_ht = p; }
    ~HtScope() { g_ht = saved; }
  } ht_scope(&ht);
  Timer total_timer;
  DevPool work;   // freed at the end of the factorization
  UnitBuf gram_units, elim_units;   // launch lists of the tcgen05 path
  ScratchPool level_scratch;
  struct Ev {
    cudaEvent_t e = nullptr;
    ~Ev() { if (e) cudaEventDestroy(e); }
  } ev_run_holder;
  CK(cudaEventCreateWithFlags(&ev_run_holder.e, cudaEventDisableTiming));
  cudaEvent_t ev_run = ev_run_holder.e;
  // Pinned host buffers reused from level to level (grown, never shrunk):
  // a level's box ranks, its final active counts and positions (read by the
  // host as soon as the last colour's IDs are done, while the GPU still runs
  // that colour's products and the host sets up the next level), and its
  // status word and refinement residuals (read one level later, once the
  // GPU has finished the level).
  PinnedPool pinned;
  DevSlots pools;   // the levels' Schur pools, by level parity
  enum { kPinRun = 0, kPinCurN = 1, kPinActPos = 2, kPinStatus = 3, kPinNs = 4, kPinStatusIds = 5 };
  Ev ev_ids_holder;   // the last colour's IDs of a level are final
  CK(cudaEventCreateWithFlags(&ev_ids_holder.e, cudaEventDisableTiming));
  cudaEvent_t ev_ids = ev_ids_holder.e;
  // a level whose status and statistics are read once its GPU work is done
  struct Pending {
    bool on = false;
    int lev = 0, nb = 0, colours = 0, nprox = 0, ns_rmax = 0;
    size_t current = 0;
    int64_t sum_a = 0, sum_s = 0, max_a = 0, max_r = 0, pool = 0;
    std::vector<int> r;                 // per box
  } pend;
  H->d_perm = H->mem.get<int>((size_t)n);
  CK(cudaMemcpyAsync(H->d_perm, tree->d_perm, n * sizeof(int), cudaMemcpyDeviceToDevice, st));
  double* soa = work.get<double>((size_t)n * 8);
  launch_permute_geometry(pts, nrm, w, tree->d_perm, n, soa, st);
  CK(cudaGetLastError());
  Geometry g{soa, soa + n, soa + 2 * n, soa + 3 * n, soa + 4 * n, soa + 5 * n, soa + 6 * n,
             soa + 7 * n, k, H->eta};
  // mixed path: near-field and proxy kernel values in fp32 from split copies
  if (H->fp32) g.f = launch_split_geometry(soa, n, work.get<float>((size_t)n * 10), st);
  int* d_status = work.get<int>(1);
  CK(cudaMemsetAsync(d_status, 0, sizeof(int), st));

  std::ostringstream js;
  js << "{\"n\": " << n << ", \"k\": " << k << ", \"eta\": " << H->eta << ", \"eps\": " << eps
     << ", \"precision\": \"" << (H->fp32 ? "mixed" : "fp64") << "\", \"id_method\": \"" << (H->gram ? "gram" : "householder") << "\", \"nlevels\": " << T.nlevels
     << ", \"levels\": [";
  std::unique_ptr<LevelState> prev;
  int root_level = 1;
  bool first_level = true;
  // events around each level's GPU work, alternating by level parity (a
  // level's pair is read while the next level runs)
  Ev lev_t0[2], lev_t1[2];
  for (int q = 0; q < 2; ++q) {
    CK(cudaEventCreate(&lev_t0[q].e));
    CK(cudaEventCreate(&lev_t1[q].e));
  }
  // the previous level's status word, refinement statistics and stats entry;
  // called after a stream synchronisation, when that level's work is done
  auto finish_pending = [&]() {
    if (!pend.on) return;
    pend.on = false;
    const int status = *pinned.get<int>(kPinStatus, 1);
    std::string msg;
    if (int code = status_to_code(status, msg))
      throw Error(code, msg + " (level " + std::to_string(pend.lev) + ")");
    int ns_boxes = 0, ns_fallback = 0;
    double ns_worst = 0.0;
    if (pend.ns_rmax >= kNsMin) {
      const unsigned long long* errs = pinned.get<unsigned long long>(kPinNs, (size_t)pend.nb);
      for (int e = 0; e < pend.nb; ++e) {
        if (pend.r[e] < kNsMin || pend.r[e] > pend.ns_rmax) continue;
        double v;
        std::memcpy(&v, &errs[e], sizeof(v));
        ++ns_boxes;
        ns_worst = std::max(ns_worst, v);
        if (!(v <= opt.xrr_refine_tol)) ++ns_fallback;
      }
    }
    float lms = 0.f;
    CK(cudaEventElapsedTime(&lms, lev_t0[pend.lev & 1].e, lev_t1[pend.lev & 1].e));
    if (opt.verbose)
      std::fprintf(stderr, "[fmmlu] level %d: boxes %d colours %d current %zu sum_a %lld sum_s %lld max_a %lld max_r %lld pool %.1f MB %.1f ms; refined inverses %d (worst residual %.1e, fp64 again %d)\n",
                   pend.lev, pend.nb, pend.colours, pend.current, (long long)pend.sum_a,
                   (long long)pend.sum_s, (long long)pend.max_a, (long long)pend.max_r,
                   pend.pool * 16.0 / 1e6, (double)lms, ns_boxes, ns_worst, ns_fallback);
    js << (first_level ? "" : ", ") << "{\"level\": " << pend.lev << ", \"boxes\": " << pend.nb
       << ", \"colours\": " << pend.colours << ", \"n_proxy\": " << pend.nprox
       << ", \"current\": " << pend.current
       << ", \"sum_a\": " << pend.sum_a << ", \"sum_s\": " << pend.sum_s << ", \"max_a\": " << pend.max_a
       << ", \"max_r\": " << pend.max_r << ", \"refined_inverses\": " << ns_boxes
       << ", \"refine_fallbacks\": " << ns_fallback << ", \"ms\": " << lms << "}";
    first_level = false;
  };
  for (int lev = T.nlevels - 1; lev >= 2; --lev) {
    const HLevel& HL = T.levels.at(lev);
    CK(cudaEventRecord(lev_t0[lev & 1].e, st));
    std::unique_ptr<LevelState> L;
    {
      HostTimer mt(&HostTimes::make_level);
      L = make_level(T, lev, prev.get(), &HL, st, &pools);
    }
    const auto setup0 = std::chrono::steady_clock::now();
    auto sub0 = setup0;
    // stop rule: any level box with active far DOFs?
    const int nb = (int)HL.boxes.size();
    bool far_any = false;
    for (int r = 0; r < nb && !far_any; ++r) {
      int64_t closed = L->a0[L->cidx.at(HL.boxes[r])];
      for (int j = HL.nbeg[r]; j < HL.nbeg[r] + HL.ncnt[r]; ++j) closed += L->a0[L->cidx.at(HL.nlist[j])];
      if (L->total() - closed > 0) far_any = true;
    }
    if (!far_any) {
      root_level = lev;
      prev = std::move(L);
      break;
    }
    // proxy points of this level's spheres (Sec. 5.2)
    const double hlev = T.side / (double)(1 << lev);
    const int nprox = proxy_count_for(opt, k, opt.proxy_radius_factor * 0.86602540378443864676 * hlev,
                                      eps_id);
    // descriptors in elimination order
    std::vector<BoxDesc> desc(nb);
    std::vector<int> nlist, qlist;
    std::vector<int64_t> pairtab, qpair;
    int64_t ptab_size = 0, qpair_size = 0;
    std::vector<int> seg_start;
    int64_t arena = 0, iarena = 0;
    const double hreal = T.side / (double)(1 << lev);
    for (int e = 0; e < nb; ++e) {
      int r = HL.order[e];
      int B = HL.boxes[r];
      const HBox& hb = T.boxes[B];
      BoxDesc& d = desc[e];
      std::memset(&d, 0, sizeof(d));
      d.cur = L->cidx.at(B);
      d.a = L->a0[d.cur];
      d.nbeg = (int)nlist.size();
      d.ncnt = HL.ncnt[r];
      d.nmax = 0;
      for (int j = HL.nbeg[r]; j < HL.nbeg[r] + HL.ncnt[r]; ++j) {
        int c = L->cidx.at(HL.nlist[j]);
        nlist.push_back(c);
        d.nmax += L->a0[c];
      }
      d.qbeg = (int)qlist.size();
      d.qcnt = HL.qcnt[r];
      d.qmax = 0;
      for (int j = HL.qbeg[r]; j < HL.qbeg[r] + HL.qcnt[r]; ++j) {
        int c = L->cidx.at(HL.qlist[j]);
        qlist.push_back(c);
        d.qmax += L->a0[c];
      }
      d.mmax = 2 * d.qmax + 2 * nprox;
      d.h = hreal;
      d.cx = T.corner[0] + ((double)hb.cx + 0.5) * hreal;
      d.cy = T.corner[1] + ((double)hb.cy + 0.5) * hreal;
      d.cz = T.corner[2] + ((double)hb.cz + 0.5) * hreal;
      // block offsets are looked up below, in parallel over the boxes
      d.pairtab = ptab_size;
      ptab_size += (int64_t)(d.ncnt + 1) * (d.ncnt + 1);
      d.qpair = qpair_size;
      qpair_size += 2 * (int64_t)d.qcnt;
      int64_t a = d.a, nm = d.nmax;
      d.G1_off = arena; arena += a * (a + nm);
      d.G3_off = arena; arena += (a + nm) * a;
      d.T_off = arena; arena += a * a;
      d.Xinv_off = arena; arena += a * a;
      d.idx_off = iarena; iarena += (a + nm) + a;
      if (e == 0 || HL.colour[HL.order[e - 1]] != HL.colour[r]) seg_start.push_back(e);
    }
    seg_start.push_back(nb);
    ht.setup_desc += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - sub0).count();
    sub0 = std::chrono::steady_clock::now();
    // pool offsets of the blocks between the boxes of each closed
    // neighbourhood {B} u N(B), and of the blocks (q, B), (B, q) for q in Q(B)
    pairtab.resize((size_t)ptab_size);
    qpair.resize((size_t)qpair_size);
    parallel_for(nb, [&](int64_t e0, int64_t e1) {
      std::vector<int> cn;
      for (int64_t e = e0; e < e1; ++e) {
        const BoxDesc& d = desc[e];
        cn.assign(1, d.cur);
        for (int j = 0; j < d.ncnt; ++j) cn.push_back(nlist[d.nbeg + j]);
        int64_t o = d.pairtab;
        for (int x : cn)
          for (int y : cn) pairtab[o++] = L->pair.find(x, y);
        o = d.qpair;
        for (int j = 0; j < d.qcnt; ++j) {
          const int c = qlist[d.qbeg + j];
          qpair[o++] = L->pair.find(c, d.cur);
          qpair[o++] = L->pair.find(d.cur, c);
        }
      }
    });
    ht.setup_pairs += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - sub0).count();
    sub0 = std::chrono::steady_clock::now();
    // per-colour scratch offsets (reset at each colour start)
    int64_t rows_max = 0, M_max = 0, W_max = 0;
    for (size_t sgi = 0; sgi + 1 < seg_start.size(); ++sgi) {
      int64_t ro = 0, mo = 0, wo = 0;
      for (int e = seg_start[sgi]; e < seg_start[sgi + 1]; ++e) {
        BoxDesc& d = desc[e];
        d.rows_off = ro; ro += 3 * (int64_t)(d.qmax + d.nmax);
        d.M_off = mo; mo += (int64_t)d.mmax * d.a;
        d.W_off = wo; wo += (int64_t)(d.a + d.nmax) * d.a;
      }
      rows_max = std::max(rows_max, ro);
      M_max = std::max(M_max, mo);
      W_max = std::max(W_max, wo);
    }
    ScratchPool& lw = level_scratch;   // level scratch, reused across levels
    lw.reset();
    double2* d_arena = H->mem.get<double2>((size_t)arena);
    int* d_iarena = H->mem.get<int>((size_t)iarena);
    H->arena_bytes += arena * 16 + iarena * 4;
    LevelDev LD;
    LD.desc = lw.up(desc, st);
    BoxRun* d_run = lw.get<BoxRun>((size_t)nb);
    BoxRun* h_run = opt.schur_emulation == 1 ? pinned.get<BoxRun>(kPinRun, (size_t)nb) : nullptr;
    CK(cudaMemsetAsync(d_run, 0, nb * sizeof(BoxRun), st));
    LD.run = d_run;
    LD.nlist = lw.up(nlist, st);
    LD.qlist = lw.up(qlist, st);
    LD.pairtab = lw.up(pairtab, st);
    LD.qpair = lw.up(qpair, st);
    LD.cur_n = L->d_cur_n;
    LD.cur_off = L->d_cur_off;
    LD.cur_a0 = L->d_cur_a0;
    LD.act_dof = L->d_act_dof;
    LD.act_pos = L->d_act_pos;
    LD.delta = L->d_pool;
    LD.rows = lw.get<int>((size_t)rows_max);
    LD.Mbuf = H->fp32 ? (void*)lw.get<float2>((size_t)M_max) : (void*)lw.get<double2>((size_t)M_max);
    LD.Wbuf = lw.get<double2>((size_t)W_max);
    LD.arena = d_arena;
    LD.iarena = d_iarena;
    LD.n_proxy = nprox;
    LD.proxy_factor = opt.proxy_radius_factor;
    LD.eps = eps_id;
    LD.status = d_status;
    // refinement of X_RR^{-1} (tcgen05 path): per colour an X_RR copy and a
    // product scratch of a^2 each per box
    int ns_rmax = 0;
    unsigned char* d_ns_skip = nullptr;   // boxes that skip the third refinement step
    if (opt.schur_emulation == 1 && opt.xrr_refine_tol >= 0.0) {   // the tcgen05 path
      for (int r = kNsMin; r <= 4096; r += 8)
        if (gj32_cluster_size(r) > 0) ns_rmax = r; else break;
    }
    {
      std::vector<int64_t> nso(nb, 0);
      int64_t ns_max = 0;
      if (ns_rmax >= kNsMin)
        for (size_t sgi = 0; sgi + 1 < seg_start.size(); ++sgi) {
          int64_t o = 0;
          for (int e = seg_start[sgi]; e < seg_start[sgi + 1]; ++e) {
            nso[e] = o;
            o += 2 * (int64_t)desc[e].a * desc[e].a;
          }
          ns_max = std::max(ns_max, o);
        }
      LD.nsbuf = ns_rmax >= kNsMin ? lw.get<double2>((size_t)ns_max) : nullptr;
      LD.ns_off = lw.up(nso, st);
      LD.ns_err = lw.get<unsigned long long>((size_t)nb);
      d_ns_skip = lw.get<unsigned char>((size_t)nb);
      LD.ns_rmax = ns_rmax;
    }
    // CPQR plan per colour: boxes share the co-resident CTAs in proportion to
    // their work (rows x a^2); colours with many boxes use one CTA per box.
    struct ColPlan { int pbeg = 0, np = 0; int64_t scratch = 0; bool dist = false; };
    // colours whose largest box exceeds the pivoted Cholesky's shared memory
    // take the Householder QR
    std::vector<char> gram_col(seg_start.size(), 0);
    if (use_gram) {
      int dev = 0, optin = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      for (size_t sgi = 0; sgi + 1 < seg_start.size(); ++sgi) {
        int amax = 1;
        for (int e = seg_start[sgi]; e < seg_start[sgi + 1]; ++e) amax = std::max(amax, desc[e].a);
        gram_col[sgi] = pchol_smem(amax) <= (size_t)optin ? 1 : 0;
      }
    }
    std::vector<ColPlan> cplan(seg_start.size());
    std::vector<CpqrPart> parts;
    int64_t cpqr_scratch = 0;
    for (size_t sgi = 0; sgi + 1 < seg_start.size(); ++sgi) {
      int b0 = seg_start[sgi], cnt = seg_start[sgi + 1] - b0;
      int amax = 1;
      for (int e = b0; e < b0 + cnt; ++e) amax = std::max(amax, desc[e].a);
      int cap = cpqr_dist_capacity(amax, H->fp32);
      ColPlan& cp = cplan[sgi];
      if (gram_col[sgi] || opt.cpqr_single || cap <= 0 || 2 * cnt > cap) continue;
      double wsum = 0;
      std::vector<double> wgt(cnt);
      for (int e = 0; e < cnt; ++e) {
        const BoxDesc& d = desc[b0 + e];
        wgt[e] = (double)d.mmax * d.a * d.a;
        wsum += wgt[e];
      }
      std::vector<int> P(cnt);
      int tot = 0;
      for (int e = 0; e < cnt; ++e) {
        int pmax = std::max(1, std::min(H->fp32 ? 32 : 160, desc[b0 + e].mmax / 64));
        P[e] = std::max(1, std::min(pmax, (int)std::floor(cap * wgt[e] / wsum)));
        tot += P[e];
      }
      while (tot > cap) {
        int big = (int)(std::max_element(P.begin(), P.end()) - P.begin());
        if (P[big] <= 1) break;
        --P[big];
        --tot;
      }
      if (tot > cap) continue;
      cp.dist = true;
      cp.pbeg = (int)parts.size();
      cp.np = tot;
      int64_t off = 0;
      for (int e = 0; e < cnt; ++e) {
        for (int c = 0; c < P[e]; ++c) parts.push_back(CpqrPart{b0 + e, c, P[e], 0, off});
        off += (int64_t)cpqr_dist_scratch_bytes(P[e], desc[b0 + e].a, H->fp32);
      }
      cp.scratch = off;
      cpqr_scratch = std::max(cpqr_scratch, off);
    }
    // Gauss-Jordan plan: CTAs in proportion to a^3 (r is only known on the
    // device; a bounds it), at least 16 columns per CTA.
    std::vector<ColPlan> gplan(seg_start.size());
    int64_t gj_scratch = 0;
    for (size_t sgi = 0; sgi + 1 < seg_start.size(); ++sgi) {
      int b0 = seg_start[sgi], cnt = seg_start[sgi + 1] - b0;
      int amax = 1;
      for (int e = b0; e < b0 + cnt; ++e) amax = std::max(amax, desc[e].a);
      int cap = gj_dist_capacity(amax);
      ColPlan& gp = gplan[sgi];
      if (opt.cpqr_single || cap <= 0 || 2 * cnt > cap || amax < 32) continue;
      double wsum = 0;
      for (int e = b0; e < b0 + cnt; ++e) wsum += std::pow((double)desc[e].a, 3.0);
      std::vector<int> P(cnt);
      int tot = 0;
      for (int e = 0; e < cnt; ++e) {
        double a3 = std::pow((double)desc[b0 + e].a, 3.0);
        int pmax = std::max(1, desc[b0 + e].a / 16);
        P[e] = std::max(1, std::min(pmax, (int)std::floor(cap * a3 / wsum)));
        tot += P[e];
      }
      while (tot > cap) {
        int big = (int)(std::max_element(P.begin(), P.end()) - P.begin());
        if (P[big] <= 1) break;
        --P[big];
        --tot;
      }
      if (tot > cap) continue;
      gp.dist = true;
      gp.pbeg = (int)parts.size();
      gp.np = tot;
      int64_t off = 0;
      for (int e = 0; e < cnt; ++e) {
        for (int q = 0; q < P[e]; ++q) parts.push_back(CpqrPart{b0 + e, q, P[e], 0, off});
        off += (int64_t)gj_dist_scratch_bytes(desc[b0 + e].a);
      }
      gp.scratch = off;
      gj_scratch = std::max(gj_scratch, off);
    }
    // Gram form of the ID: per colour digit slices, exponents and G/R blocks;
    // pivoted-Cholesky CTAs in proportion to a^3 with >= 8 columns per CTA,
    // co-resident (cooperative) when the colour fits, else one CTA per box.
    // G = M^H M on tcgen05 (default) or on the mma.sync path (schur_emulation 2)
    const bool gram_tc = opt.schur_emulation != 2;
    std::vector<GramBoxHost> gbh(use_gram ? nb : 0);
    std::vector<TcBoxHost> gtb(use_gram && gram_tc ? nb : 0);
    std::vector<ColPlan> pplan(seg_start.size());
    int64_t gr_slices = 0, gr_expo = 0, gr_g = 0, pc_scratch = 0;
    if (use_gram) {
      for (size_t sgi = 0; sgi + 1 < seg_start.size(); ++sgi) {
        if (!gram_col[sgi]) continue;
        int b0 = seg_start[sgi], cnt = seg_start[sgi + 1] - b0;
        int64_t so = 0, eo = 0, go = 0, tso = 0, teo = 0;
        int amax = 1;
        for (int e = b0; e < b0 + cnt; ++e) {
          plan_gram_box(desc[e].a, desc[e].mmax, H->fp32, so, eo, go, gbh[e]);
          if (gram_tc) {
            plan_tc_box(desc[e].a, desc[e].a, desc[e].mmax, H->fp32 ? 4 : 7, tso, teo, gtb[e]);
            // G = M^H M: the rows of A and the columns of B are both the
            // columns of M, so one exponent per column serves both sides
            gtb[e].eb_off = gtb[e].ea_off;
          }
          amax = std::max(amax, desc[e].a);
        }
        gr_slices = std::max(gr_slices, gram_tc ? tso : 2 * so);   // bytes
        gr_expo = std::max(gr_expo, gram_tc ? teo : eo);
        gr_g = std::max(gr_g, go);
        const int cap = pchol_capacity(amax);
        std::vector<int> P(cnt, 1);
        int tot = cnt;
        ColPlan& pp = pplan[sgi];
        pp.dist = cnt <= cap;
        if (pp.dist) {
          double wsum = 0;
          for (int e = b0; e < b0 + cnt; ++e) wsum += std::pow((double)desc[e].a, 3.0);
          tot = 0;
          for (int e = 0; e < cnt; ++e) {
            const int a = desc[b0 + e].a;
            const int pmax = std::max(1, (a + 7) / 8);   // >= 8 columns per CTA
            P[e] = std::max(1, std::min(pmax, (int)std::floor(cap * std::pow((double)a, 3.0) /
                                                              std::max(wsum, 1.0))));
            tot += P[e];
          }
          while (tot > cap) {
            int big = (int)(std::max_element(P.begin(), P.end()) - P.begin());
            if (P[big] <= 1) break;
            --P[big];
            --tot;
          }
        }
        pp.pbeg = (int)parts.size();
        pp.np = tot;
        int64_t off = 0;
        for (int e = 0; e < cnt; ++e) {
          for (int c = 0; c < P[e]; ++c) parts.push_back(CpqrPart{b0 + e, c, P[e], 0, off});
          off += (int64_t)pchol_scratch_bytes(P[e]);
        }
        pp.scratch = off;
        pc_scratch = std::max(pc_scratch, off);
      }
    }
    std::vector<char> gram_box(nb, 0);
    for (size_t sgi = 0; sgi + 1 < seg_start.size(); ++sgi)
      for (int e = seg_start[sgi]; e < seg_start[sgi + 1]; ++e) gram_box[e] = gram_col[sgi];
    GramBoxHost* d_gbh = use_gram ? lw.up(gbh, st) : nullptr;
    TcBoxHost* d_gtb = use_gram && gram_tc ? lw.up(gtb, st) : nullptr;
    // split-K accumulator of the Gram products: 4 int64 per entry of each box's G
    std::vector<int64_t> gx_off(nb, 0), gx_col_off(seg_start.size(), 0), gx_col_len(seg_start.size(), 0);
    int64_t gx_max = 1;
    if (use_gram && gram_tc)
      for (size_t sgi = 0; sgi + 1 < seg_start.size(); ++sgi) {
        int64_t o = 0;
        for (int e = seg_start[sgi]; e < seg_start[sgi + 1]; ++e) {
          gx_off[e] = o;
          o += 4 * (int64_t)desc[e].a * desc[e].a;
        }
        gx_col_len[sgi] = o;
        gx_max = std::max(gx_max, o);
      }
    unsigned long long* d_gx = use_gram && gram_tc ? lw.get<unsigned long long>((size_t)gx_max) : nullptr;
    const int64_t* d_gx_off = use_gram && gram_tc ? lw.up(gx_off, st) : nullptr;
    void* d_gr_slices = use_gram ? (void*)lw.get<unsigned char>((size_t)gr_slices) : nullptr;
    int* d_gr_expo = use_gram ? lw.get<int>((size_t)gr_expo) : nullptr;
    double2* d_gr_g = use_gram ? lw.get<double2>((size_t)gr_g) : nullptr;
    unsigned char* d_pc_scratch = use_gram ? lw.get<unsigned char>((size_t)pc_scratch) : nullptr;
    // Schur update on tensor cores: per-box slice scratch (bounds), per colour
    std::vector<OzBoxHost> ozb(nb);
    std::vector<int64_t> oz_seg_slices(seg_start.size(), 0), oz_seg_expo(seg_start.size(), 0);
    int64_t oz_slices = 0, oz_expo = 0;
    const bool use_oz = opt.schur_emulation != 0;
    const bool use_tc = opt.schur_emulation == 1;    // tcgen05; 2 = mma.sync
    // tcgen05 elimination products (G1, G3, W, Schur): operand bounds per box
    std::vector<TcBoxHost> tcb(use_tc ? nb : 0);
    int64_t tc_slices = 0, tc_expo = 0;
    if (use_tc) {
      for (size_t sgi = 0; sgi + 1 < seg_start.size(); ++sgi) {
        int64_t so = 0, eo = 0;
        for (int e = seg_start[sgi]; e < seg_start[sgi + 1]; ++e)
          plan_tc_box(desc[e].a + desc[e].nmax, desc[e].a + desc[e].nmax, desc[e].a, 7, so, eo,
                      tcb[e]);
        tc_slices = std::max(tc_slices, so);
        tc_expo = std::max(tc_expo, eo);
      }
    }
    TcBoxHost* d_tcb = use_tc ? lw.up(tcb, st) : nullptr;
    void* d_tc_slices = use_tc ? (void*)lw.get<unsigned char>((size_t)tc_slices) : nullptr;
    int* d_tc_expo = use_tc ? lw.get<int>((size_t)tc_expo) : nullptr;
    if (use_oz && !use_tc) {
      for (size_t sgi = 0; sgi + 1 < seg_start.size(); ++sgi) {
        int64_t so = 0, eo = 0;
        for (int e = seg_start[sgi]; e < seg_start[sgi + 1]; ++e)
          plan_oz_box(desc[e].a, desc[e].nmax, so, eo, ozb[e]);
        oz_slices = std::max(oz_slices, so);
        oz_expo = std::max(oz_expo, eo);
      }
    }
    const bool use_mma = use_oz && !use_tc;
    OzBoxHost* d_ozb = use_mma ? lw.up(ozb, st) : nullptr;
    void* d_oz_slices = use_mma ? (void*)lw.get<uint16_t>((size_t)oz_slices) : nullptr;
    int* d_oz_expo = use_mma ? lw.get<int>((size_t)oz_expo) : nullptr;
    ht.setup_plans += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - sub0).count();
    sub0 = std::chrono::steady_clock::now();
    CpqrPart* d_parts = lw.up(parts, st);
    unsigned char* d_cpqr_scratch = lw.get<unsigned char>((size_t)cpqr_scratch);
    unsigned char* d_gj_scratch = lw.get<unsigned char>((size_t)gj_scratch);
    ht.setup += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() -
                                                          setup0).count();
    // the set-up above ran on the host while the GPU finished the previous
    // level and merged its Schur blocks into this level's pool
    stream_wait(st);
    prev.reset();
    finish_pending();
    for (size_t sgi = 0; sgi + 1 < seg_start.size(); ++sgi) {
      int b0 = seg_start[sgi], cnt = seg_start[sgi + 1] - b0;
      int amax = 1, mmax = 1, nmaxm = 0;
      for (int e = b0; e < b0 + cnt; ++e) {
        amax = std::max(amax, desc[e].a);
        mmax = std::max(mmax, desc[e].mmax);
        nmaxm = std::max(nmaxm, desc[e].nmax);
      }
      launch_gather_rows(LD, b0, cnt, st);
      CK(launch_assemble_id(LD, g, b0, cnt, mmax, H->fp32, st));
      if (gram_col[sgi]) {
        if (gram_tc) {
          // Gram tiles from a (exact); the k range (split into chunks whose
          // exact int64 sums add up in gx) from the row bound m_max
          std::vector<TcBoxSize> bs(cnt);
          for (int e = 0; e < cnt; ++e) bs[e] = TcBoxSize{desc[b0 + e].a, 0, 0, 0, desc[b0 + e].mmax};
          std::vector<TcUnit> units;
          TcPlan pl;
          int fin0 = 0;
          auto gram_product = [&](int chunk) {
            units.clear();
            tc_plan(kTcGram, bs, units, pl, chunk);
            fin0 = (int)units.size();
            for (int e = 0; e < cnt; ++e) units.push_back(TcUnit{e, 0, 0, 0});
            gram_units.upload(units, st);
            CK(cudaMemsetAsync(d_gx + gx_col_off[sgi], 0,
                               (size_t)gx_col_len[sgi] * sizeof(unsigned long long), st));
            launch_tc_planned(kTcGram, LD, b0, d_gtb + b0, d_gr_slices, d_gr_expo, d_gbh, d_gr_g,
                              H->fp32, gram_units.d, pl, st, d_gx, d_gx_off);
          };
          gram_product(gram_chunk_for(opt, bs, H->fp32, st, gram_product));
          launch_gram_finalize(LD, b0, gram_units.d + fin0, cnt, amax, d_gtb + b0, d_gr_expo, d_gbh,
                               d_gr_g, d_gx, d_gx_off, H->fp32, st);
        } else
          launch_gram(LD, b0, cnt, d_gbh, d_gr_slices, d_gr_expo, d_gr_g, amax, mmax, H->fp32, st);
        CK(cudaGetLastError());
        CK(cudaMemsetAsync(d_pc_scratch, 0, (size_t)pplan[sgi].scratch, st));
        CK(launch_pchol(LD, d_parts + pplan[sgi].pbeg, pplan[sgi].np, d_pc_scratch, d_gbh,
                        d_gr_g, amax, pplan[sgi].dist, st));
      } else if (cplan[sgi].dist) {
        CK(cudaMemsetAsync(d_cpqr_scratch, 0, (size_t)cplan[sgi].scratch, st));
        CK(launch_cpqr_dist(LD, d_parts + cplan[sgi].pbeg, cplan[sgi].np, d_cpqr_scratch, amax,
                            H->fp32, st));
      } else {
        launch_cpqr(LD, b0, cnt, H->fp32, amax, st);
      }
      // exact sizes of this colour's boxes (the ID fixed s and r): the tcgen05
      // launches get exact unit lists instead of bounds
      TcPlan epl[8];
      int ns_off0 = 0, ns_cnt = 0, ns_rmax_c = 0;   // boxes whose X_RR^{-1} is refined
      if (use_tc) {
        CK(cudaMemcpyAsync(h_run + b0, d_run + b0, cnt * sizeof(BoxRun), cudaMemcpyDeviceToHost,
                           st));
        if (sgi + 2 == seg_start.size()) {
          // the last colour's IDs complete the level's active counts and
          // positions: copy them now, ahead of the colour's products
          CK(cudaMemcpyAsync(pinned.get<int>(kPinCurN, L->cur.size()), L->d_cur_n,
                             L->cur.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
          CK(cudaMemcpyAsync(pinned.get<int>(kPinActPos, L->act_pos.size()), L->d_act_pos,
                             L->act_pos.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
          CK(cudaMemcpyAsync(pinned.get<int>(kPinStatusIds, 1), d_status, sizeof(int),
                             cudaMemcpyDeviceToHost, st));
          CK(cudaEventRecord(ev_ids, st));
        }
        CK(cudaEventRecord(ev_run, st));
      }
      // the elimination blocks need no plan: the GPU assembles them while the
      // host waits for the ranks and plans the products
      CK(launch_assemble_elim(LD, g, b0, cnt, amax, nmaxm, H->fp32, st));
      if (use_tc) {
        {
          HostTimer wt(&HostTimes::wait);
          CK(cudaEventSynchronize(ev_run));
        }
        HostTimer pt(&HostTimes::plan);
        std::vector<TcBoxSize> bs(cnt);
        for (int e = 0; e < cnt; ++e) {
          const BoxRun& q = h_run[b0 + e];
          bs[e] = TcBoxSize{desc[b0 + e].a, q.s, q.r, q.n, 0, ns_rmax};
        }
        std::vector<TcUnit> units;
        for (int w : {kTcG1, kTcG3, kTcW, kTcSchur, kTcXrr}) tc_plan(w, bs, units, epl[w]);
        if (ns_rmax >= kNsMin) {
          for (int w : {kTcNsY, kTcNsX}) tc_plan(w, bs, units, epl[w]);
          ns_off0 = (int)units.size();
          for (int e = 0; e < cnt; ++e) {
            const int r = h_run[b0 + e].r;
            if (r >= kNsMin && r <= ns_rmax) {
              units.push_back(TcUnit{e, 0, 0, 0});
              ns_rmax_c = std::max(ns_rmax_c, r);
            }
          }
          ns_cnt = (int)units.size() - ns_off0;
        }
        elim_units.upload(units, st);
      }
      const int kskip = use_tc ? kTcInnerMin : use_oz ? kOzInnerMin : 0;
      // the fp64 FMA products take the boxes whose inner dimension is below
      // kskip; with the tcgen05 path (kskip = 1) only empty products are
      // left for G1, G3, W and the Schur update
      const bool fma_left = kskip != 1;
      if (fma_left) {
        launch_gemm_g1(LD, b0, cnt, amax, nmaxm, st, kskip);
        launch_gemm_g3(LD, b0, cnt, amax, nmaxm, st, kskip);
      }
      if (use_tc) {
        launch_tc_planned(kTcG1, LD, b0, d_tcb + b0, d_tc_slices, d_tc_expo, nullptr, nullptr,
                          false, elim_units.d, epl[kTcG1], st);
        launch_tc_planned(kTcG3, LD, b0, d_tcb + b0, d_tc_slices, d_tc_expo, nullptr, nullptr,
                          false, elim_units.d, epl[kTcG3], st);
      } else if (use_oz) {
        launch_oz_elim_gemms(LD, b0, cnt, d_ozb + b0, d_oz_slices, d_oz_expo, amax, nmaxm, 0, st);
        launch_oz_elim_gemms(LD, b0, cnt, d_ozb + b0, d_oz_slices, d_oz_expo, amax, nmaxm, 1, st);
      }
      // (X_RR of a box with no skeleton, s = 0, is still copied here)
      launch_gemm_xrr(LD, b0, cnt, amax, st, use_tc ? kTcInnerMin : 0);
      if (use_tc)
        launch_tc_planned(kTcXrr, LD, b0, d_tcb + b0, d_tc_slices, d_tc_expo, nullptr, nullptr,
                          false, elim_units.d, epl[kTcXrr], st);
      // X_RR^{-1}: boxes with kNsMin <= r <= ns_rmax by an fp32 inverse over a
      // thread-block cluster and two Newton-Schulz steps on the tensor cores
      // (boxes whose residual stays above 1e-9 are inverted again in fp64);
      // the other boxes by fp64 Gauss-Jordan
      bool ns_done = false;
      if (ns_cnt > 0) {
        const int P = gj32_cluster_size(ns_rmax_c);
        cudaError_t eg = P > 0 ? launch_gj32(LD, b0, elim_units.d + ns_off0, ns_cnt, ns_rmax_c, P, st)
                               : cudaErrorNotSupported;
        if (eg == cudaSuccess) {
          launch_xrr_inverse(LD, b0, cnt, amax, st, kNsMin, ns_rmax);
          auto ns = [&](int w) {
            launch_tc_planned(w, LD, b0, d_tcb + b0, d_tc_slices, d_tc_expo, nullptr, nullptr, false,
                              elim_units.d, epl[w], st);
          };
          // up to three steps. A step's residual e (max |I - X_RR X|) bounds
          // the next iterate's by (r e)^2: boxes whose second-step residual
          // gives (r e)^2 <= min(tol, eps / 100) skip the third step; for the
          // others the third step's residual must be <= tol, leaving the
          // result below ~1e-12 for r <= 640 (else fp64 Gauss-Jordan again)
          ns(kTcNsY);
          ns(kTcNsX);
          CK(cudaMemsetAsync(LD.ns_err + b0, 0, (size_t)cnt * sizeof(unsigned long long), st));
          ns(kTcNsY);
          ns(kTcNsX);
          launch_ns_flag(LD, b0, elim_units.d + ns_off0, ns_cnt,
                         std::min(opt.xrr_refine_tol, 1e-2 * eps), d_ns_skip, st);
          {
            LevelDev LD3 = LD;
            LD3.ns_skip = d_ns_skip;
            launch_tc_planned(kTcNsY, LD3, b0, d_tcb + b0, d_tc_slices, d_tc_expo, nullptr, nullptr,
                              false, elim_units.d, epl[kTcNsY], st);
            launch_tc_planned(kTcNsX, LD3, b0, d_tcb + b0, d_tc_slices, d_tc_expo, nullptr, nullptr,
                              false, elim_units.d, epl[kTcNsX], st);
          }
          launch_ns_fallback(LD, b0, elim_units.d + ns_off0, ns_cnt, amax, opt.xrr_refine_tol, st);
          ns_done = true;
        } else if (eg != cudaErrorNotSupported) {
          CK(eg);
        }
      }
      if (!ns_done) {
        if (gplan[sgi].dist) {
          CK(cudaMemsetAsync(d_gj_scratch, 0, (size_t)gplan[sgi].scratch, st));
          CK(launch_gj_dist(LD, d_parts + gplan[sgi].pbeg, gplan[sgi].np, d_gj_scratch, amax, st));
        } else {
          launch_xrr_inverse(LD, b0, cnt, amax, st);
        }
      }
      if (fma_left) launch_gemm_w(LD, b0, cnt, amax, nmaxm, st, kskip);
      if (use_tc)
        launch_tc_planned(kTcW, LD, b0, d_tcb + b0, d_tc_slices, d_tc_expo, nullptr, nullptr,
                          false, elim_units.d, epl[kTcW], st);
      else if (use_oz)
        launch_oz_elim_gemms(LD, b0, cnt, d_ozb + b0, d_oz_slices, d_oz_expo, amax, nmaxm, 2, st);
      if (fma_left) launch_schur_update(LD, b0, cnt, amax, nmaxm, st, kskip);
      if (use_tc)
        launch_tc_planned(kTcSchur, LD, b0, d_tcb + b0, d_tc_slices, d_tc_expo, nullptr, nullptr,
                          false, elim_units.d, epl[kTcSchur], st);
      else if (use_oz)
        launch_oz_schur(LD, b0, cnt, d_ozb + b0, d_oz_slices, d_oz_expo, amax, nmaxm, st);
      CK(cudaGetLastError());
    }
    std::vector<BoxRun> run;
    int* h_status = pinned.get<int>(kPinStatus, 1);
    if (use_tc) {
      // counts and positions as copied after the last colour's IDs; the GPU
      // may still run that colour's products. The status word and the
      // refinement residuals are read with the next level.
      {
        HostTimer wt(&HostTimes::wait);
        CK(cudaEventSynchronize(ev_ids));
      }
      std::string msg;   // the IDs must have succeeded before their ranks are used
      if (int code = status_to_code(*pinned.get<int>(kPinStatusIds, 1), msg))
        throw Error(code, msg + " (level " + std::to_string(lev) + ")");
      run.assign(h_run, h_run + nb);
      const int* pcn = pinned.get<int>(kPinCurN, L->cur.size());
      const int* pap = pinned.get<int>(kPinActPos, L->act_pos.size());
      L->cur_n.assign(pcn, pcn + L->cur.size());
      L->act_pos.assign(pap, pap + L->act_pos.size());
      CK(cudaMemcpyAsync(h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
      if (ns_rmax >= kNsMin)
        CK(cudaMemcpyAsync(pinned.get<unsigned long long>(kPinNs, (size_t)nb), LD.ns_err,
                           (size_t)nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    } else {
      run = ddownload(d_run, (size_t)nb, st);
      *h_status = ddownload(d_status, 1, st)[0];
      std::string msg;
      if (int code = status_to_code(*h_status, msg))
        throw Error(code, msg + " (level " + std::to_string(lev) + ")");
      L->cur_n = ddownload(L->d_cur_n, L->cur.size(), st);
      L->act_pos = ddownload(L->d_act_pos, L->act_pos.size(), st);
      if (ns_rmax >= kNsMin) {
        std::vector<unsigned long long> errs = ddownload(LD.ns_err, (size_t)nb, st);
        std::memcpy(pinned.get<unsigned long long>(kPinNs, (size_t)nb), errs.data(),
                    (size_t)nb * sizeof(unsigned long long));
      }
    }
    if (H->profile) {
      H->prof.resolve();
      const double csz = H->fp32 ? 8.0 : 16.0;
      for (int e = 0; e < nb; ++e) {
        const BoxDesc& d = desc[e];
        const BoxRun& rr = run[e];
        double a = d.a, s_ = rr.s, r_ = rr.r, n_ = rr.n;
        double m = 2.0 * rr.nq + 2.0 * nprox;
        // one kernel evaluation per entry of M, kKevalFlops real flops each
        // (besides the exponential); the outgoing and incoming rows of a pair
        // share one distance and one exp(ikr)
        H->prof.add_work("assemble_id", kKevalFlops * m * a, m * a * csz);
        if (gram_box[e]) {
          const double ns = H->fp32 ? 4.0 : 7.0, apad = std::ceil(a / 64.0) * 64.0;
          const double kt = std::ceil(m / 16.0) * 16.0;
          double pc = 4.0 * s_ * s_ * r_;
          for (int j = 0; j < rr.s; ++j) pc += 8.0 * j * (a - j - 1);
          H->prof.add_work(gram_tc ? "tc_split" : "gram_split", 0,
                           gram_tc ? a * m * (4.0 * csz + 10.0 * ns) : m * a * csz + ns * 4.0 * apad * kt);
          // bf16 tensor flops of the upper-triangle tiles: digit pairs x 4 real
          // products x 2 flops x m x a (a + 1) / 2
          const double pairs = H->fp32 ? 13.0 : 28.0;
          H->prof.add_work("gram", pairs * 8.0 * m * a * (a + 1) / 2.0,
                           ns * 4.0 * apad * kt + 16.0 * a * a, 8.0 * m * a * (a + 1) / 2.0);
          H->prof.add_work("pchol", pc, 16.0 * (a * a + a * s_ + s_ * r_));
        } else {
          double qr = 0;
          for (int j = 0; j < rr.s; ++j) qr += 18.0 * (m - j) * (a - j - 1);
          qr += 4.0 * s_ * s_ * r_;
          H->prof.add_work("cpqr", qr, m * a * csz);
        }
        if (rr.r == 0) continue;
        // G1 and G3 entries come in pairs from one kernel evaluation
        H->prof.add_work("assemble_elim", kKevalFlops * 2.0 * a * (a + n_),
                         2.0 * a * (a + n_) * 16.0);
        // complex products: 8 fp64 flops per multiply-add on the FMA path; on
        // the tensor-core path (inner dimension >= kOzInnerMin) 28 digit pairs
        // x 4 real bf16 products x 2 flops, and the digit split of the operands
        const int inner_min = use_tc ? kTcInnerMin : kOzInnerMin;
        const bool tc_s = use_oz && rr.s >= inner_min, tc_r = use_oz && rr.r >= inner_min;
        const double c_tc = 28.0 * 4.0 * 2.0;
        // split bytes per element: the operand read twice (exponent, digits), 7 digits written
        // as 2 (A side) or 3 (B side) bf16 parts
        auto split = [](double ra, double rb, double kk) {
          return ra * kk * (32.0 + 28.0) + rb * kk * (32.0 + 42.0);
        };
        H->prof.add_work(tc_s ? "gemm_g1_tc" : "gemm_g1", (tc_s ? c_tc : 8.0) * r_ * (a + n_) * s_,
                         16.0 * (s_ * r_ + 2 * a * (a + n_)), 8.0 * r_ * (a + n_) * s_);
        H->prof.add_work(tc_s ? "gemm_g3_tc" : "gemm_g3", (tc_s ? c_tc : 8.0) * (a + n_) * r_ * s_,
                         16.0 * (s_ * r_ + 2 * a * (a + n_)), 8.0 * (a + n_) * r_ * s_);
        const char* split_name = use_tc ? "tc_split" : "oz_split";
        if (tc_s) H->prof.add_work(split_name, 0, split(r_, a + n_, s_) + split(a + n_, r_, s_));
        H->prof.add_work(use_tc && tc_s ? "gemm_xrr_tc" : "gemm_xrr",
                         (use_tc && tc_s ? c_tc : 8.0) * r_ * r_ * s_,
                         16.0 * (2 * r_ * r_ + r_ * s_ + s_ * r_), 8.0 * r_ * r_ * s_);
        if (use_tc && tc_s) H->prof.add_work(split_name, 0, split(r_, r_, s_));
        if (use_tc && ns_rmax >= kNsMin && rr.r >= kNsMin && rr.r <= ns_rmax) {
          // fp32 Gauss-Jordan, then two Newton-Schulz steps (two products each)
          H->prof.add_work("xrr_inverse32", 8.0 * r_ * r_ * r_, 16.0 * 3 * r_ * r_);
          H->prof.add_work("ns_tc", 6.0 * c_tc * r_ * r_ * r_, 16.0 * 6 * 3 * r_ * r_,
                           6.0 * 8.0 * r_ * r_ * r_);
          H->prof.add_work(split_name, 0, 6.0 * split(r_, r_, r_));
        } else {
          H->prof.add_work("xrr_inverse", 8.0 * r_ * r_ * r_, 16.0 * 2 * r_ * r_);
        }
        H->prof.add_work(tc_r ? "gemm_w_tc" : "gemm_w", (tc_r ? c_tc : 8.0) * (s_ + n_) * r_ * r_,
                         16.0 * (2 * (s_ + n_) * r_ + r_ * r_), 8.0 * (s_ + n_) * r_ * r_);
        H->prof.add_work(tc_r ? "schur_tc" : "schur_update",
                         (tc_r ? c_tc : 8.0) * (s_ + n_) * (s_ + n_) * r_,
                         16.0 * (2 * (s_ + n_) * r_ + 2 * (s_ + n_) * (s_ + n_)),
                         8.0 * (s_ + n_) * (s_ + n_) * r_);
        if (tc_r) H->prof.add_work(split_name, 0, split(s_ + n_, r_, r_) + split(s_ + n_, s_ + n_, r_));
      }
    }
    // solve plan for this level: the eliminated boxes of each colour in
    // elimination order (their chunk items are built per chunk size by
    // make_solve_plan)
    int64_t sum_a = 0, sum_s = 0, max_a = 0, max_r = 0;
    for (size_t sgi = 0; sgi + 1 < seg_start.size(); ++sgi) {
      const int b0p = (int)H->sboxes.size();
      int rmax = 0, smax = 0;
      double fc = 0, bc = 0, fb = 0, bb = 0, seg_vbytes = 0;
      for (int e = seg_start[sgi]; e < seg_start[sgi + 1]; ++e) {
        const BoxDesc& d = desc[e];
        const BoxRun& rr = run[e];
        sum_a += d.a; sum_s += rr.s;
        max_a = std::max<int64_t>(max_a, d.a);
        max_r = std::max<int64_t>(max_r, rr.r);
        if (rr.r == 0) continue;
        int64_t ld3 = d.a + d.nmax;
        SolveBox sb{};
        sb.r = rr.r; sb.s = rr.s; sb.n = rr.n;
        sb.idx = d_iarena + d.idx_off;
        sb.T = d_arena + d.T_off; sb.ldT = d.a;
        sb.Xinv = d_arena + d.Xinv_off; sb.ldX = d.a;
        sb.XCR = d_arena + d.G3_off + (int64_t)rr.s * ld3; sb.ldL = (int)ld3;
        sb.XRC = d_arena + d.G1_off + rr.s; sb.ldU = d.a;
        H->sboxes.push_back(sb);
        rmax = std::max(rmax, rr.r);
        smax = std::max(smax, rr.s);
        double ec = (double)(rr.s + rr.n) * rr.r;
        double eb = (double)rr.s * rr.r + (double)rr.r * rr.r;
        fc += 8.0 * ec; bc += 16.0 * ec;
        fb += 8.0 * eb; bb += 16.0 * eb;
        seg_vbytes += 16.0 * 2.0 * (rr.r + rr.s + rr.n);
        H->factor_entries += (int64_t)rr.s * rr.r + (int64_t)rr.r * rr.r +
                             2 * (int64_t)(rr.s + rr.n) * rr.r;
      }
      const int cnt = (int)H->sboxes.size() - b0p;
      if (cnt > 0) {
        SweepSeg sg{};
        sg.b0 = b0p; sg.nb = cnt;
        sg.rmax = rmax; sg.smax = smax;
        sg.flops_c = fc; sg.bytes_c = bc; sg.flops_b = fb; sg.bytes_b = bb;
        sg.bytes_per_rhs = seg_vbytes;
        H->sseg.push_back(sg);
      }
    }
    CK(cudaEventRecord(lev_t1[lev & 1].e, st));
    pend.on = true;
    pend.lev = lev;
    pend.nb = nb;
    pend.colours = HL.ncolours;
    pend.nprox = nprox;
    pend.ns_rmax = ns_rmax;
    pend.current = L->cur.size();
    pend.sum_a = sum_a;
    pend.sum_s = sum_s;
    pend.max_a = max_a;
    pend.max_r = max_r;
    pend.pool = L->pool_size;
    pend.r.resize((size_t)nb);
    for (int e = 0; e < nb; ++e) pend.r[(size_t)e] = run[(size_t)e].r;
    prev = std::move(L);
  }
  stream_wait(st);
  finish_pending();
  // ---- root ----------------------------------------------------------------
  Timer rt;
  std::unique_ptr<LevelState> R;
  if (prev && prev->level == root_level) {
    R = std::move(prev);
  } else {
    {
      HostTimer mt(&HostTimes::make_level);
      R = make_level(T, root_level, prev.get(), nullptr, st, &pools);
    }
    stream_wait(st);
    prev.reset();
  }
  int n0 = (int)R->total();
  H->n0 = n0;
  if (n0 > 0) {
    int nc = (int)R->cur.size();
    std::vector<int> owner(n0), pos(n0);
    for (int c = 0; c < nc; ++c)
      for (int i = 0; i < R->a0[c]; ++i) { owner[R->off[c] + i] = c; pos[R->off[c] + i] = i; }
    std::vector<int64_t> pairoff((size_t)nc * nc, -1);
    for (int x = 0; x < nc; ++x)
      for (int64_t e = R->pair.start[x]; e < R->pair.start[x + 1]; ++e)
        pairoff[(size_t)x * nc + R->pair.ys[e]] = R->pair.off[e];
    DevPool rw;
    int* d_owner = rw.up(owner, st);
    int* d_pos = rw.up(pos, st);
    int64_t* d_pairoff = rw.up(pairoff, st);
    H->d_root_dofs = H->mem.up(R->act_dof, st);
    H->d_root = H->mem.get<double2>((size_t)n0 * n0);
    launch_assemble_root(g, H->d_root_dofs, d_owner, d_pos, d_pairoff, R->d_cur_a0, nc, R->d_pool,
                         n0, H->d_root, st);
    double2* wk = rw.get<double2>((size_t)n0 * H->nb_root);
    CK(launch_root_factor(H->d_root, n0, H->nb_root, wk, d_status, st, opt.schur_emulation == 1));
    CK(cudaGetLastError());
    int status = ddownload(d_status, 1, st)[0];
    std::string msg;
    if (int code = status_to_code(status, msg)) throw Error(code, msg + " (root)");
    if (H->profile) {
      H->prof.resolve();
      double rb = 0;
      for (int i0 = 0; i0 < n0; i0 += H->nb_root) {
        double r_ = std::min(H->nb_root, n0 - i0), later = n0 - i0 - r_;
        H->prof.add_work("root_diag", 8.0 * r_ * r_ * r_, 16.0 * 2 * r_ * r_);
        if (later > 0) {
          const bool tcr = opt.schur_emulation == 1 && r_ >= kTcInnerMin;
          const double c = tcr ? 28.0 * 4.0 * 2.0 : 8.0;
          H->prof.add_work(tcr ? "root_w_tc" : "root_w", c * later * r_ * r_,
                           16.0 * (2 * later * r_ + r_ * r_), 8.0 * later * r_ * r_);
          H->prof.add_work(tcr ? "root_schur_tc" : "root_schur", c * later * later * r_,
                           16.0 * (2 * later * later + 2 * later * r_), 8.0 * later * later * r_);
        }
        rb += 1;
      }
      H->prof.add_work("assemble_root", 0, 16.0 * n0 * (double)n0);
    }
    H->factor_entries += (int64_t)n0 * n0;
  }
  double root_ms = rt.ms();
  H->plans[H->chunk0] = make_solve_plan(H, H->chunk0, st);
  {
    // FNV-1a over the solve's structure: the key of tuned solve settings
    uint64_t hs = 1469598103934665603ull;
    auto mix = [&](int64_t v) {
      for (int i = 0; i < 8; ++i) { hs ^= (uint64_t)(v >> (8 * i)) & 0xffu; hs *= 1099511628211ull; }
    };
    mix(n); mix(n0);
    for (const SolveBox& sb : H->sboxes) { mix(sb.r); mix(sb.s); mix(sb.n); }
    for (const SweepSeg& sg : H->sseg) { mix(sg.b0); mix(sg.nb); }
    H->shape_key = hs;
  }
  stream_wait(st);
  double tot_ms = total_timer.ms();
  if (opt.verbose)
    std::fprintf(stderr, "[fmmlu] root level %d n0 %d %.1f ms; factor %.1f ms; m_f %.1f MB\n",
                 root_level, n0, root_ms, tot_ms, H->factor_entries * 16.0 / 1e6);
  js << "], \"root_level\": " << root_level << ", \"n0\": " << n0 << ", \"root_ms\": " << root_ms
     << ", \"factor_ms\": " << tot_ms << ", \"factor_bytes\": " << H->factor_entries * 16
     << ", \"arena_bytes\": " << H->arena_bytes << ", \"eliminated_boxes\": " << H->sboxes.size()
     << ", \"colour_segments\": " << H->sseg.size() << ", \"host_ms\": {\"alloc\": " << ht.alloc
     << ", \"allocs\": " << ht.allocs << ", \"release\": " << ht.release
     << ", \"wait\": " << ht.wait << ", \"make_level\": " << ht.make_level
     << ", \"plan\": " << ht.plan << ", \"level_setup\": " << ht.setup
     << ", \"setup_desc\": " << ht.setup_desc << ", \"setup_pairs\": " << ht.setup_pairs
     << ", \"setup_plans\": " << ht.setup_plans << "}}";
  H->stats = js.str();
}

// ---------------------------------------------------------------------------
// solve runtime: plans per chunk size, work vectors per (nrhs, direction,
// stream, chunk), CUDA graphs of the sweeps, and the chunk-size tuner
// ---------------------------------------------------------------------------

constexpr size_t kMaxSolveCtx = 4;
constexpr int kTuneChunks[] = {32, 64, 128, 256};

std::shared_ptr<SolvePlan> get_plan(const fmmlu_handle* H, int chunk, cudaStream_t st) {
  auto it = H->plans.find(chunk);
  if (it != H->plans.end()) return it->second;
  auto P = make_solve_plan(H, chunk, st);
  H->plans[chunk] = P;
  return P;
}

size_t counter_bytes(const fmmlu_handle* H, int nrhs) {
  return (H->sboxes.size() * (size_t)nrhs + 1) * sizeof(int);
}

void alloc_ctx(const fmmlu_handle* H, SolveCtx& c) {
  const int64_t n = H->n;
  if (c.tcp) {
    c.tslices = c.mem.get<unsigned char>((size_t)c.tcp->slice_bytes);
    c.texpo = c.mem.get<int>((size_t)c.tcp->expo_ints);
  }
  c.v = c.mem.get<double2>((size_t)n * c.nrhs);
  c.part = c.mem.get<double2>((size_t)c.plan->part_max * c.nrhs);
  c.cnt = c.mem.get<int>(counter_bytes(H, c.nrhs) / sizeof(int));
  if (H->n0 > 0) {
    c.vr = c.mem.get<double2>((size_t)H->n0 * c.nrhs);
    c.z = c.mem.get<double2>((size_t)H->n0 * c.nrhs);
    c.rscr = c.mem.get<unsigned char>(root_solve_scratch_bytes(H->n0, H->nb_root, c.nrhs));
  }
}

// forward sweep, root, backward sweep on the permuted vectors c.v (in place)
void run_sweeps(const fmmlu_handle* H, const SolveCtx& c, cudaStream_t st) {
  const SolvePlan& P = *c.plan;
  const int64_t n = H->n, pst = P.part_max;
  const TcSolvePlan* tp = c.tcp.get();
  LevelDev Ls;   // context of the tensor-core C products
  std::memset(&Ls, 0, sizeof(Ls));
  if (tp) {
    Ls.desc = P.d_desc;
    Ls.run = P.d_run;
    Ls.status = P.d_status;
    Ls.sbox = P.d_boxes;
    Ls.sv = c.v;
    Ls.sn = n;
    Ls.snrhs = c.nrhs;
    Ls.spart = c.part;
    Ls.spst = pst;
  }
  CK(cudaMemsetAsync(c.cnt, 0, counter_bytes(H, c.nrhs), st));
  for (size_t q = 0; q < P.segs.size(); ++q) {
    const SweepSeg& sg = P.segs[q];
    launch_sweep(P.d_boxes, P.d_items, sg, c.v, n, c.nrhs, false, c.adjoint, c.part, pst, st,
                 c.cnt, tp != nullptr);
    if (tp) {
      launch_tc_planned(c.adjoint ? kTcSvCA : kTcSvC, Ls, sg.b0, tp->d_tbC + sg.b0, c.tslices,
                        c.texpo, nullptr, nullptr, false, tp->d_units, tp->plC[q], st);
      launch_copy_z(P.d_boxes, sg.b0, sg.nb, sg.rmax, c.v, n, c.nrhs, c.part, pst, st);
    }
  }
  if (H->n0 > 0) {
    launch_root_gather(c.v, H->d_root_dofs, H->n0, n, c.nrhs, c.vr, st);
    CK(launch_root_solve(H->d_root, H->n0, H->nb_root, c.vr, c.z, c.rscr, c.nrhs, c.adjoint, st));
    launch_root_scatter(c.vr, H->d_root_dofs, H->n0, n, c.nrhs, c.v, st);
  }
  // t slots start at zero (a box with an empty C gets no product)
  if (tp) CK(cudaMemsetAsync(c.part, 0, sizeof(double2) * (size_t)pst * c.nrhs, st));
  for (size_t q = P.segs.size(); q-- > 0;) {
    const SweepSeg& sg = P.segs[q];
    if (tp)
      launch_tc_planned(c.adjoint ? kTcSvTA : kTcSvT, Ls, sg.b0, tp->d_tbT + sg.b0, c.tslices,
                        c.texpo, nullptr, nullptr, false, tp->d_units, tp->plT[q], st);
    launch_sweep(P.d_boxes, P.d_items, sg, c.v, n, c.nrhs, true, c.adjoint, c.part, pst, st,
                 c.cnt, tp != nullptr);
  }
}

// Record the sweeps of c into a CUDA graph on the handle's own capture stream
// (the caller's stream may be the legacy default stream, which cannot be
// captured); the graph is launched on the caller's stream.
void capture_ctx(const fmmlu_handle* H, SolveCtx& c) {
  if (!H->cap_stream) CK(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
  prepare_solve_kernels();
  ProfScope none(nullptr);
  const int64_t l0 = launches_total();
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal));
  try {
    run_sweeps(H, c, H->cap_stream);
  } catch (...) {
    cudaStreamEndCapture(H->cap_stream, &g);
    if (g) cudaGraphDestroy(g);
    launches_add(l0 - launches_total());
    throw;
  }
  CK(cudaStreamEndCapture(H->cap_stream, &g));
  c.graph_kernels = launches_total() - l0;
  launches_add(-c.graph_kernels);
  cudaError_t e = cudaGraphInstantiate(&c.exec, g, 0);
  cudaGraphDestroy(g);
  CK(e);
}

SolveCtx* get_ctx(const fmmlu_handle* H, int nrhs, bool adjoint, cudaStream_t st, int chunk) {
  for (auto& c : H->ctxs)
    if (c->nrhs == nrhs && c->adjoint == adjoint && c->stream == st && c->plan->chunk == chunk)
      return c.get();
  if (H->ctxs.size() >= kMaxSolveCtx) {   // drop the least recently used (waits for it)
    auto lru = std::min_element(H->ctxs.begin(), H->ctxs.end(),
                                [](const std::unique_ptr<SolveCtx>& a,
                                   const std::unique_ptr<SolveCtx>& b) { return a->last < b->last; });
    H->ctxs.erase(lru);
  }
  auto c = std::make_unique<SolveCtx>();
  c->nrhs = nrhs;
  c->adjoint = adjoint;
  c->stream = st;
  c->plan = get_plan(H, chunk, st);
  if (H->solve_tc_nrhs > 0 && nrhs >= H->solve_tc_nrhs)
    c->tcp = get_tc_solve_plan(H, *c->plan, nrhs, adjoint, st);
  alloc_ctx(H, *c);
  CK(cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming));
  H->ctxs.push_back(std::move(c));
  return H->ctxs.back().get();
}

// Time the whole solve (both sweeps and the root) once per candidate chunk on
// the caller's right-hand sides; the fastest of three timed runs after one
// warm-up counts. Every candidate computes the same solution (only the order
// of the partial sums differs).
int tune_solve_chunk(const fmmlu_handle* H, int nrhs, bool adjoint, const double* b,
                     cudaStream_t st) {
  ProfScope none(nullptr);
  struct Ev {
    cudaEvent_t e = nullptr;
    ~Ev() { if (e) cudaEventDestroy(e); }
  } e0, e1;
  CK(cudaEventCreate(&e0.e));
  CK(cudaEventCreate(&e1.e));
  float best = INFINITY;
  int bestc = H->chunk0;
  for (int chunk : kTuneChunks) {
    SolveCtx t;
    t.nrhs = nrhs;
    t.adjoint = adjoint;
    t.plan = get_plan(H, chunk, st);
    if (H->solve_tc_nrhs > 0 && nrhs >= H->solve_tc_nrhs)
      t.tcp = get_tc_solve_plan(H, *t.plan, nrhs, adjoint, st);
    alloc_ctx(H, t);
    float tmin = INFINITY;
    for (int rep = 0; rep < 4; ++rep) {
      launch_gather_vec(reinterpret_cast<const double2*>(b), H->d_perm, H->n, nrhs, t.v, st);
      CK(cudaEventRecord(e0.e, st));
      run_sweeps(H, t, st);
      CK(cudaEventRecord(e1.e, st));
      CK(cudaEventSynchronize(e1.e));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0.e, e1.e));
      if (rep > 0) tmin = std::min(tmin, ms);
    }
    if (tmin < best) {
      best = tmin;
      bestc = chunk;
    }
  }
  return bestc;
}

int choose_chunk(const fmmlu_handle* H, int nrhs, bool adjoint, const double* b, cudaStream_t st) {
  const auto key = std::make_pair(nrhs, adjoint ? 1 : 0);
  auto it = H->chunk_for.find(key);
  if (it != H->chunk_for.end()) return it->second;
  int chunk = H->chunk0;
  if (H->autotune) {
    char hx[32];
    std::snprintf(hx, sizeof(hx), "%016llx", (unsigned long long)H->shape_key);
    const std::string tk = "solve_chunk|" + device_tag() + "|" + hx + "|nrhs=" +
                           std::to_string(nrhs) + "|adj=" + (adjoint ? "1" : "0");
    if (!tune_lookup(H->tune_cache, tk, &chunk)) chunk = tune_solve_chunk(H, nrhs, adjoint, b, st);
    tune_store(H->tune_cache, tk, chunk);
  }
  H->chunk_for[key] = chunk;
  return chunk;
}

// Algorithmic flops and bytes of one solve (both sweeps and the root) for the
// per-kernel accounting of a profiled handle.
void account_solve(const fmmlu_handle* H, const SolvePlan& plan, int nrhs, bool tc = false) {
  for (const auto& sg : plan.segs) {
    H->prof.add_work("sweep_fwd", sg.flops_b * nrhs, sg.bytes_b + sg.bytes_per_rhs * nrhs / 2);
    H->prof.add_work("sweep_bwd", sg.flops_b * nrhs, sg.bytes_b + sg.bytes_per_rhs * nrhs / 2);
    if (!tc) {
      H->prof.add_work("sweep_fwd_c", sg.flops_c * nrhs, sg.bytes_c + sg.bytes_per_rhs * nrhs / 2);
      H->prof.add_work("sweep_bwd_t", sg.flops_c * nrhs, sg.bytes_c + sg.bytes_per_rhs * nrhs / 2);
      continue;
    }
    // exact split: 28 digit pairs x 4 real products per complex multiply-add
    // (8 fp64 flops); the stored block is split on every solve (read twice,
    // 28 B of digits written and read back per entry)
    const double entries = sg.bytes_c / 16.0;
    for (const char* nm : {"sweep_c_tc", "sweep_t_tc"})
      H->prof.add_work(nm, 28.0 * sg.flops_c * nrhs, 28.0 * entries + sg.bytes_per_rhs * nrhs / 2,
                       sg.flops_c * nrhs);
    H->prof.add_work("tc_split", 0, 2.0 * entries * (32.0 + 28.0));
  }
  const int n0 = H->n0;
  for (int i0 = 0; i0 < n0; i0 += H->nb_root) {
    const double r_ = std::min(H->nb_root, n0 - i0), later = n0 - i0 - r_;
    H->prof.add_work("root_fwd", 8.0 * nrhs * (r_ * r_ + later * r_),
                     16.0 * (r_ * r_ + later * r_ + 2.0 * nrhs * (later + r_)));
    H->prof.add_work("root_bwd", 8.0 * nrhs * (later * r_ + r_ * r_),
                     16.0 * (later * r_ + r_ * r_ + nrhs * (later + 2.0 * r_)));
  }
}

// The factors live on the device that was current at fmmlu_factor; a solve
// must run with that device current.
void check_device(const fmmlu_handle* H) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev != H->device)
    throw Error(FMMLU_ERR_INVALID_ARG, "the current device (" + std::to_string(dev) +
                                           ") is not the one the factors live on (" +
                                           std::to_string(H->device) + ")");
}

void solve_impl(const fmmlu_handle* H, const double* b, double* x, int nrhs, bool adjoint,
                cudaStream_t st) {
  check_device(H);
  std::lock_guard<std::mutex> lock(H->smu);
  const int chunk = choose_chunk(H, nrhs, adjoint, b, st);
  SolveCtx* c = get_ctx(H, nrhs, adjoint, st, chunk);
  const bool graph =
      !H->profile && (H->solve_graph == 2 || (H->solve_graph == 1 && c->uses >= 1));
  ProfScope prof_scope(H->profile ? &H->prof : nullptr);
  const int64_t n = H->n;
  launch_gather_vec(reinterpret_cast<const double2*>(b), H->d_perm, n, nrhs, c->v, st);
  if (graph) {
    if (!c->exec) capture_ctx(H, *c);
    CK(cudaGraphLaunch(c->exec, st));
    launches_add(c->graph_kernels);
  } else {
    run_sweeps(H, *c, st);
  }
  launch_scatter_vec(c->v, H->d_perm, n, nrhs, reinterpret_cast<double2*>(x), st);
  CK(cudaGetLastError());
  CK(cudaEventRecord(c->done, st));
  ++c->uses;
  c->last = ++H->tick;
  if (H->profile) {
    CK(cudaStreamSynchronize(st));
    H->prof.resolve();
    account_solve(H, *c->plan, nrhs, c->tcp != nullptr);
  }
}

// ---------------------------------------------------------------------------
// GMRES preconditioned by the stored factors (Sec. 7): A M^{-1} u = b,
// x = M^{-1} u, M^{-1} = fmmlu_solve, A = the dense on-the-fly product.
// ---------------------------------------------------------------------------

struct GmresResult {
  int iters = 0;
  double relres = 0.0;     // true ||b - A x|| / ||b|| at the end
  bool converged = false;  // the Givens estimate reached tol
};

void gmres_impl(const fmmlu_handle* H, const double* pts, const double* nrm, const double* wts,
                const double2* b, double2* x, double tol, int restart, int maxiter,
                cudaStream_t st, GmresResult& res) {
  const int64_t n = H->n;
  DevPool mem;
  std::vector<int> iota((size_t)n);
  std::iota(iota.begin(), iota.end(), 0);
  int* d_id = mem.up(iota, st);
  double* soa = mem.get<double>((size_t)n * 8);
  launch_permute_geometry(pts, nrm, wts, d_id, n, soa, st);
  Geometry g{soa, soa + n, soa + 2 * n, soa + 3 * n, soa + 4 * n, soa + 5 * n, soa + 6 * n,
             soa + 7 * n, H->k, H->eta};
  const int ldh = kKrMaxBasis;
  double2* V = mem.get<double2>((size_t)n * kKrMaxBasis);
  double2* w = mem.get<double2>((size_t)n);
  double2* u = mem.get<double2>((size_t)n);
  double2* z = mem.get<double2>((size_t)n);
  double2* Hm = mem.get<double2>((size_t)ldh * kKrMaxRestart);
  double2* hc = mem.get<double2>(kKrMaxBasis);
  double2* gv = mem.get<double2>(kKrMaxBasis);
  double2* yv = mem.get<double2>(kKrMaxBasis);
  double2* nr = mem.get<double2>(kKrMaxBasis);
  double* cs = mem.get<double>(kKrMaxRestart);
  double2* sn = mem.get<double2>(kKrMaxRestart);
  double* scal = mem.get<double>(2);
  double* est = mem.get<double>(2);
  double2* part = mem.get<double2>((size_t)kr_blocks(n) * kKrMaxBasis);
  struct Pinned {
    double* p = nullptr;
    ~Pinned() { if (p) cudaFreeHost(p); }
  } hest;
  CK(cudaMallocHost(&hest.p, 2 * sizeof(double)));
  auto read_est = [&]() {
    CK(cudaMemcpyAsync(hest.p, est, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  };
  auto norm2_into = [&](const double2* v) {   // nr[0] = (||v||^2, 0)
    launch_kr_dots(v, n, 1, v, n, part, nr, nullptr, st);
  };
  auto apply_a = [&](const double2* v, double2* y) { launch_matvec(g, n, v, y, 1, st); };
  auto apply_minv = [&](const double2* v, double2* y) {
    solve_impl(H, reinterpret_cast<const double*>(v), reinterpret_cast<double*>(y), 1, false, st);
  };
  CK(cudaMemsetAsync(x, 0, (size_t)n * sizeof(double2), st));
  norm2_into(b);
  launch_kr_start(nr, gv, kKrMaxBasis, scal, est, st);
  read_est();
  const double bnorm = hest.p[0];
  res = GmresResult{};
  if (!(bnorm > 0.0)) {
    res.converged = true;
    return;
  }
  int its = 0;
  while (its < maxiter && !res.converged) {
    // r = b - A x, beta = ||r||, V[:, 0] = r / beta
    apply_a(x, u);
    launch_kr_residual(w, b, u, n, st);
    norm2_into(w);
    launch_kr_start(nr, gv, kKrMaxBasis, scal, est, st);
    read_est();
    if (hest.p[0] <= tol * bnorm) {
      res.converged = true;
      break;
    }
    launch_kr_scale(V, w, scal, n, st);
    const int m = std::min(restart, maxiter - its);
    CK(cudaMemsetAsync(Hm, 0, sizeof(double2) * (size_t)ldh * kKrMaxRestart, st));
    int jd = 0;
    for (int j = 0; j < m; ++j) {
      apply_minv(V + (int64_t)j * n, z);
      apply_a(z, w);
      double2* Hj = Hm + (int64_t)j * ldh;
      for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
        launch_kr_dots(V, n, j + 1, w, n, part, hc, Hj, st);
        launch_kr_update(w, V, n, j + 1, hc, n, st);
      }
      norm2_into(w);
      launch_kr_givens(Hm, ldh, j, nr, cs, sn, gv, scal, est, st);
      launch_kr_scale(V + (int64_t)(j + 1) * n, w, scal, n, st);
      ++its;
      jd = j + 1;
      read_est();
      if (hest.p[0] <= tol * bnorm) res.converged = true;
      if (res.converged || hest.p[1] == 0.0) break;
    }
    launch_kr_trisolve(Hm, ldh, jd, gv, yv, st);
    launch_kr_combine(u, V, n, jd, yv, n, st);
    apply_minv(u, z);
    launch_kr_add(x, z, n, st);
  }
  // true residual of the result
  apply_a(x, u);
  launch_kr_residual(w, b, u, n, st);
  norm2_into(w);
  launch_kr_start(nr, gv, kKrMaxBasis, scal, est, st);
  read_est();
  res.iters = its;
  res.relres = hest.p[0] / bnorm;
}

inline size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// Work-space layout of fmmlu_solve_noalloc for one (nrhs, direction): the
// permuted vectors (16 nrhs N bytes), the root's two vectors (16 nrhs n0
// each) and its partial sums, the backward sweep's partial sums (16 nrhs p,
// p = part_max of the solve plan: the largest sum over one colour's boxes of
// r x (column chunks + 1)) and one counter per eliminated box and right-hand
// side; each piece starts on a 256-byte boundary. The plan is the one of an
// earlier solve with this nrhs and direction (its tuned chunk size), else the
// factorization's own: both exist already, nothing is built here.
struct NoallocLayout {
  std::shared_ptr<SolvePlan> plan;
  size_t bv = 0, br = 0, bp = 0, bs = 0, bc = 0, need = 0;
};

NoallocLayout noalloc_layout(const fmmlu_handle* h, int nrhs, bool adj) {
  NoallocLayout L;
  {
    std::lock_guard<std::mutex> lock(h->smu);
    int chunk = h->chunk0;
    auto it = h->chunk_for.find(std::make_pair(nrhs, adj ? 1 : 0));
    if (it != h->chunk_for.end()) chunk = it->second;
    auto pit = h->plans.find(chunk);
    L.plan = pit != h->plans.end() ? pit->second : h->plans.at(h->chunk0);
  }
  L.bv = round256((size_t)16 * h->n * nrhs);
  L.br = round256((size_t)16 * h->n0 * nrhs);
  L.bp = round256(root_solve_scratch_bytes(h->n0, h->nb_root, nrhs));
  L.bs = round256((size_t)16 * nrhs * L.plan->part_max);
  L.bc = round256(counter_bytes(h, nrhs));
  L.need = L.bv + 2 * L.br + L.bp + L.bs + L.bc;
  return L;
}

}  // namespace

// ---------------------------------------------------------------------------
// exported C ABI
// ---------------------------------------------------------------------------

namespace {
int guard(const std::function<void()>& f) {
  try {
    f();
    g_err.clear();
    return FMMLU_OK;
  } catch (const Error& e) {
    g_err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return FMMLU_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return FMMLU_ERR_CUDA;
  } catch (...) {
    g_err = "unknown error";
    return FMMLU_ERR_CUDA;
  }
}
}  // namespace

extern "C" {

int fmmlu_default_opts(fmmlu_opts* opts) {
  if (!opts) { g_err = "opts is NULL"; return FMMLU_ERR_INVALID_ARG; }
  default_opts(opts);
  return FMMLU_OK;
}

const char* fmmlu_last_error(void) { return g_err.c_str(); }

int fmmlu_build_tree(const double* points, int64_t n, const fmmlu_opts* opts, void* stream,
                     fmmlu_tree** out) {
  return guard([&] {
    if (!points || !out || n < 1) throw Error(FMMLU_ERR_INVALID_ARG, "null argument or n < 1");
    if (n > (int64_t)1 << 30) throw Error(FMMLU_ERR_LIMIT, "n above 2^30");
    *out = nullptr;
    fmmlu_opts o = checked_opts(opts);
    cudaStream_t st = (cudaStream_t)stream;
    auto t = std::make_unique<fmmlu_tree>();
    t->opts = o;
    std::string msg;
    if (int rc = gpu_build_tree(points, n, o.leaf_size, t->T, &t->d_perm, msg, o.verbose, st))
      throw Error(rc, "tree: " + msg);
    *out = t.release();
  });
}

int fmmlu_factor(const fmmlu_tree* tree, const double* points, const double* normals,
                 const double* weights, double k, double eps, const fmmlu_opts* opts,
                 void* stream, fmmlu_handle** out) {
  return guard([&] {
    if (!tree || tree->magic != kTreeMagic || !points || !normals || !weights || !out)
      throw Error(FMMLU_ERR_INVALID_ARG, "null argument or not a tree");
    if (!(k > 0.0) || !std::isfinite(k)) throw Error(FMMLU_ERR_INVALID_ARG, "k must be positive");
    if (!(eps > 0.0 && eps < 1.0)) throw Error(FMMLU_ERR_INVALID_ARG, "eps must lie in (0, 1)");
    *out = nullptr;
    fmmlu_opts o = checked_opts(opts ? opts : &tree->opts);
    auto H = std::make_unique<fmmlu_handle>();
    factor_impl(tree, points, normals, weights, k, eps, o, (cudaStream_t)stream, H.get());
    *out = H.release();
  });
}

int fmmlu_solve(const fmmlu_handle* h, const double* b, double* x, int nrhs, void* stream) {
  return guard([&] {
    if (!h || h->magic != kHandleMagic || !b || !x || nrhs < 1)
      throw Error(FMMLU_ERR_INVALID_ARG, "null argument, not a handle, or nrhs < 1");
    solve_impl(h, b, x, nrhs, false, (cudaStream_t)stream);
  });
}

int fmmlu_solve_adjoint(const fmmlu_handle* h, const double* b, double* x, int nrhs,
                        void* stream) {
  return guard([&] {
    if (!h || h->magic != kHandleMagic || !b || !x || nrhs < 1)
      throw Error(FMMLU_ERR_INVALID_ARG, "null argument, not a handle, or nrhs < 1");
    solve_impl(h, b, x, nrhs, true, (cudaStream_t)stream);
  });
}

int fmmlu_matvec(int64_t n, const double* points, const double* normals, const double* weights,
                 double k, double eta, const double* v, double* y, int nrhs, void* stream) {
  return guard([&] {
    if (n < 1 || !points || !normals || !weights || !v || !y || nrhs < 1)
      throw Error(FMMLU_ERR_INVALID_ARG, "null argument, n < 1 or nrhs < 1");
    if (v == y) throw Error(FMMLU_ERR_INVALID_ARG, "y must not alias v");
    cudaStream_t st = (cudaStream_t)stream;
    DevPool w;
    std::vector<int> iota((size_t)n);
    std::iota(iota.begin(), iota.end(), 0);
    int* d_id = w.up(iota, st);
    double* soa = w.get<double>((size_t)n * 8);
    launch_permute_geometry(points, normals, weights, d_id, n, soa, st);
    Geometry g{soa, soa + n, soa + 2 * n, soa + 3 * n, soa + 4 * n, soa + 5 * n, soa + 6 * n,
               soa + 7 * n, k, std::isnan(eta) ? k : eta};
    launch_matvec(g, n, reinterpret_cast<const double2*>(v), reinterpret_cast<double2*>(y), nrhs,
                  st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  });
}

int fmmlu_gmres(const fmmlu_handle* h, const double* points, const double* normals,
                const double* weights, const double* b, double* x, int nrhs, double tol,
                int restart, int maxiter, int* iters, double* relres, void* stream) {
  return guard([&] {
    if (!h || h->magic != kHandleMagic || !points || !normals || !weights || !b || !x ||
        nrhs < 1)
      throw Error(FMMLU_ERR_INVALID_ARG, "null argument, not a handle, or nrhs < 1");
    if (b == x) throw Error(FMMLU_ERR_INVALID_ARG, "x must not alias b");
    if (!(tol > 0.0 && tol < 1.0)) throw Error(FMMLU_ERR_INVALID_ARG, "tol must lie in (0, 1)");
    if (restart < 1 || restart > kKrMaxRestart)
      throw Error(FMMLU_ERR_INVALID_ARG, "restart must lie in [1, 64]");
    if (maxiter < 1) throw Error(FMMLU_ERR_INVALID_ARG, "maxiter must be >= 1");
    check_device(h);
    cudaStream_t st = (cudaStream_t)stream;
    bool all = true;
    for (int c = 0; c < nrhs; ++c) {
      GmresResult r;
      gmres_impl(h, points, normals, weights,
                 reinterpret_cast<const double2*>(b) + (int64_t)c * h->n,
                 reinterpret_cast<double2*>(x) + (int64_t)c * h->n, tol, restart, maxiter, st, r);
      if (iters) iters[c] = r.iters;
      if (relres) relres[c] = r.relres;
      all = all && r.converged;
    }
    if (!all)
      throw Error(FMMLU_ERR_NOT_CONVERGED,
                  "GMRES did not reach tol within maxiter steps (x holds the last iterate)");
  });
}

int fmmlu_plane_waves(int64_t n, const double* points, const double* weights, double k,
                      const double* dirs, int m, double* b, void* stream) {
  return guard([&] {
    if (n < 1 || !points || !weights || !dirs || !b || m < 1)
      throw Error(FMMLU_ERR_INVALID_ARG, "null argument, n < 1 or m < 1");
    if (!(k > 0.0) || !std::isfinite(k)) throw Error(FMMLU_ERR_INVALID_ARG, "k must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    for (int m0 = 0; m0 < m; m0 += 65535)
      launch_plane_waves(points, weights, n, k, dirs, m0, std::min(65535, m - m0),
                         reinterpret_cast<double2*>(b) + (int64_t)m0 * n, st);
    CK(cudaGetLastError());
  });
}

int fmmlu_backscatter(int64_t n, const double* points, const double* normals,
                      const double* weights, double k, double eta, const double* dirs, int m,
                      const double* x, double* R, void* stream) {
  return guard([&] {
    if (n < 1 || !points || !normals || !weights || !dirs || !x || !R || m < 1)
      throw Error(FMMLU_ERR_INVALID_ARG, "null argument, n < 1 or m < 1");
    if (!(k > 0.0) || !std::isfinite(k)) throw Error(FMMLU_ERR_INVALID_ARG, "k must be positive");
    cudaStream_t st = (cudaStream_t)stream;
    DevPool w;
    const int mb = std::min(m, 65535);
    double2* part = w.get<double2>((size_t)backscatter_blocks(n) * mb);
    for (int m0 = 0; m0 < m; m0 += mb)
      launch_backscatter(points, normals, weights, n, k, std::isnan(eta) ? k : eta, dirs, m0,
                         std::min(mb, m - m0),
                         reinterpret_cast<const double2*>(x) + (int64_t)m0 * n, part,
                         reinterpret_cast<double2*>(R), st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));   // the partial sums are freed on return
  });
}

int fmmlu_sonar_sweep(const fmmlu_handle* h, const double* points, const double* normals,
                      const double* weights, const double* dirs, int m, int batch, double* R,
                      void* stream) {
  return guard([&] {
    if (!h || h->magic != kHandleMagic || !points || !normals || !weights || !dirs || !R ||
        m < 1 || batch < 1)
      throw Error(FMMLU_ERR_INVALID_ARG, "null argument, not a handle, m < 1 or batch < 1");
    check_device(h);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = h->n;
    const int bs = std::min(std::min(batch, m), 1024);
    DevPool w;
    double2* b = w.get<double2>((size_t)n * bs);
    double2* part = w.get<double2>((size_t)backscatter_blocks(n) * bs);
    for (int m0 = 0; m0 < m; m0 += bs) {
      const int c = std::min(bs, m - m0);
      launch_plane_waves(points, weights, n, h->k, dirs + 3 * (int64_t)m0, 0, c, b, st);
      solve_impl(h, reinterpret_cast<const double*>(b), reinterpret_cast<double*>(b), c, false,
                 st);
      launch_backscatter(points, normals, weights, n, h->k, h->eta, dirs + 3 * (int64_t)m0, 0,
                         c, b, part, reinterpret_cast<double2*>(R) + m0, st);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));   // the work arrays are freed on return
  });
}

int fmmlu_stats(const fmmlu_handle* h, char* json, size_t cap) {
  if (!h || h->magic != kHandleMagic) { g_err = "not a handle"; return FMMLU_ERR_INVALID_ARG; }
  std::string s = h->stats;
  if (!s.empty() && s.back() == '}') {
    s.pop_back();
    s += ", \"profile\": " + std::string(h->profile ? "true" : "false") +
         ", \"noalloc_bytes\": {\"solve\": " + std::to_string(noalloc_layout(h, 1, false).need) +
         ", \"adjoint\": " + std::to_string(noalloc_layout(h, 1, true).need) + "}" +
         ", \"kernels\": " + h->prof.json() + "}";
  }
  if (json && cap > 0) {
    size_t m = std::min(cap - 1, s.size());
    std::memcpy(json, s.data(), m);
    json[m] = 0;
  }
  return (int)s.size();
}

int64_t fmmlu_tree_describe(const fmmlu_tree* t, int64_t* out, int64_t cap) {
  if (!t || t->magic != kTreeMagic) { g_err = "not a tree"; return FMMLU_ERR_INVALID_ARG; }
  const TreeHost& T = t->T;
  std::vector<int64_t> v;
  v.push_back(T.n);
  v.push_back((int64_t)T.boxes.size());
  v.push_back(T.nlevels);
  for (const HBox& b : T.boxes) {
    v.push_back(b.level); v.push_back(b.cx); v.push_back(b.cy); v.push_back(b.cz);
    v.push_back(b.start); v.push_back(b.end); v.push_back(b.parent);
    v.push_back((int64_t)b.kids.size());
  }
  for (int p : T.perm) v.push_back(p);
  for (int l = 2; l < T.nlevels; ++l) {
    const HLevel& L = T.levels.at(l);
    for (size_t r = 0; r < L.boxes.size(); ++r) {
      v.push_back(L.colour[r]);
      v.push_back(L.ncnt[r]);
      for (int j = L.nbeg[r]; j < L.nbeg[r] + L.ncnt[r]; ++j) v.push_back(L.nlist[j]);
      v.push_back(L.qcnt[r]);
      for (int j = L.qbeg[r]; j < L.qbeg[r] + L.qcnt[r]; ++j) v.push_back(L.qlist[j]);
    }
  }
  if (out) std::memcpy(out, v.data(), sizeof(int64_t) * (size_t)std::min<int64_t>(cap, (int64_t)v.size()));
  return (int64_t)v.size();
}

int64_t fmmlu_kernel_launches(void) { return launches_total(); }

int fmmlu_profile_reset(const fmmlu_handle* h) {
  if (!h || h->magic != kHandleMagic) { g_err = "not a handle"; return FMMLU_ERR_INVALID_ARG; }
  h->prof.reset();
  return FMMLU_OK;
}

void fmmlu_free(void* p) {
  if (!p) return;
  uint32_t m;
  std::memcpy(&m, p, sizeof(m));
  if (m == kTreeMagic) {
    auto* t = static_cast<fmmlu_tree*>(p);
    t->magic = 0;
    delete t;
  } else if (m == kHandleMagic) {
    auto* h = static_cast<fmmlu_handle*>(p);
    h->magic = 0;
    delete h;
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Solve without allocating. Some callers cannot call cudaMalloc while they
// solve: an application whose device memory is handed out entirely by its
// own pool allocator (a cudaMalloc would fail or bypass the pool), or a
// latency-critical loop that must not pay the device-wide synchronisation of
// cudaFree. For them the work vectors of a solve live in one fixed device
// array that is part of this library. Every GPU that loads the library holds
// the array until the process exits. The host cannot use the array's name as
// a device address, so the address is looked up once per device, with that
// device current, by cudaGetSymbolAddress on the first call.
// ---------------------------------------------------------------------------

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FMMLU_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kNoallocMaxDevices] = {};

unsigned char* noalloc_scratch_for_current_device() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices)
    throw Error(FMMLU_ERR_LIMIT, "device ordinal above 63 for the fixed work array");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" int fmmlu_solve_noalloc(const fmmlu_handle* h, const double* b, double* x, int nrhs,
                                   int adjoint, void* stream) {
  return guard([&] {
    if (!h || h->magic != kHandleMagic || !b || !x || nrhs < 1)
      throw Error(FMMLU_ERR_INVALID_ARG, "null argument, not a handle, or nrhs < 1");
    check_device(h);
    cudaStream_t st = (cudaStream_t)stream;
    const bool adj = adjoint != 0;
    const NoallocLayout L = noalloc_layout(h, nrhs, adj);
    if (L.need > (size_t)FMMLU_NOALLOC_SCRATCH_BYTES)
      throw Error(FMMLU_ERR_LIMIT,
                  "fmmlu_solve_noalloc needs " + std::to_string(L.need) +
                      " bytes of work space; the fixed array holds " +
                      std::to_string((size_t)FMMLU_NOALLOC_SCRATCH_BYTES));
    unsigned char* base = noalloc_scratch_for_current_device();
    const int64_t n = h->n;
    SolveCtx c;   // views into the fixed array; owns nothing
    c.nrhs = nrhs;
    c.adjoint = adj;
    c.plan = L.plan;
    c.v = reinterpret_cast<double2*>(base);
    c.vr = reinterpret_cast<double2*>(base + L.bv);
    c.z = reinterpret_cast<double2*>(base + L.bv + L.br);
    c.rscr = base + L.bv + 2 * L.br;
    c.part = reinterpret_cast<double2*>(base + L.bv + 2 * L.br + L.bp);
    c.cnt = reinterpret_cast<int*>(base + L.bv + 2 * L.br + L.bp + L.bs);
    // a profiled handle times these launches too and waits for them
    ProfScope prof_scope(h->profile ? &h->prof : nullptr);
    launch_gather_vec(reinterpret_cast<const double2*>(b), h->d_perm, n, nrhs, c.v, st);
    run_sweeps(h, c, st);
    launch_scatter_vec(c.v, h->d_perm, n, nrhs, reinterpret_cast<double2*>(x), st);
    CK(cudaGetLastError());
    if (h->profile) {
      CK(cudaStreamSynchronize(st));
      std::lock_guard<std::mutex> lock(h->smu);
      h->prof.resolve();
      account_solve(h, *L.plan, nrhs);
    }
  });
}
