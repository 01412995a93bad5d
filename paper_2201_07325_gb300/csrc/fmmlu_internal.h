// Internal declarations shared by the FMM-LU CUDA translation units.
//
// Layout conventions (device):
//  * points are Morton-sorted; DOF i is the i-th sorted point. Coordinates are
//    stored SoA: px, py, pz, nx, ny, nz, w, sqrt(w) (float64).
//  * complex128 is double2 (x = re, y = im); complex64 is float2.
//  * every dense block is column-major.
//  * "current boxes" of a level: the boxes of that level plus all coarser
//    leaves. Each has a level-start active list act0 (DOF ids) and a current
//    active subset given by positions into act0 (act_pos, first cur_n used).
//  * Schur updates are kept per ordered pair of current boxes (X, Y) as a dense
//    a0(X) x a0(Y) block (leading dimension a0(X)) indexed by act0 positions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace fmmlu {

constexpr double kPi = 3.14159265358979323846;
constexpr double kGoldenAngle = 2.39996322972865332223;  // pi (3 - sqrt 5)

// device status bits (kernels never trap; they set bits and return)
enum StatusBits : int {
  kStatusSingular = 1,
  kStatusNonfinite = 2,
  kStatusBound = 4,      // an internal size bound was exceeded
  kStatusTimeout = 8,    // a bounded inter-CTA wait gave up
};

// fp32 copies for kernel entries evaluated in single precision (mixed path):
// each coordinate as a high part (its fp32 rounding) and a low part (the
// rest, rounded), so that the difference of two points is accurate to fp32
// relative to the difference itself, however close the points are
struct GeometryF {
  const float* xh; const float* yh; const float* zh;
  const float* xl; const float* yl; const float* zl;
  const float* nx; const float* ny; const float* nz;
  const float* sw;
};

struct Geometry {        // sorted SoA copies of the inputs
  const double* px; const double* py; const double* pz;
  const double* nx; const double* ny; const double* nz;
  const double* w;  const double* sw;
  double k, eta;
  GeometryF f{};         // null unless the single-precision copies were made
};

// one per box processed at a level (host-built)
struct BoxDesc {
  int cur;          // current-box index of B
  int a;            // actives at level start
  int nbeg, ncnt;   // N boxes: nlist[nbeg .. nbeg + ncnt) (current indices)
  int qbeg, qcnt;   // Q boxes: qlist[...]
  int nmax;         // sum of a0 over N boxes
  int qmax;         // sum of a0 over Q boxes
  int mmax;         // 2 qmax + 2 n_proxy
  int pad_;
  double cx, cy, cz, h;   // centre and side of B
  int64_t pairtab;  // offset of the (1+ncnt)^2 table of Delta offsets over
                    // cn = [B, N...] (row-major [x][y]), -1 = no block
  int64_t qpair;    // offset of 2*qcnt Delta offsets: (Delta(C,B), Delta(B,C))
  int64_t rows_off; // int scratch: qdof,qpos,qloc (3 qmax), ndof,npos,nloc (3 nmax)
  int64_t M_off;    // ID matrix scratch (mmax x a), complex units of the ID type
  int64_t W_off;    // Schur scratch ((a + nmax) x a), ld a + nmax
  int64_t G1_off;   // factor arena: a x (a + nmax), ld a   rows [S|R], cols [S|N|R]
  int64_t G3_off;   // factor arena: (a + nmax) x a, ld a + nmax  rows [S|N|R], cols [S|R]
  int64_t T_off;    // factor arena: s x r, ld a
  int64_t Xinv_off; // factor arena: r x r, ld a
  int64_t idx_off;  // int arena: [R | S | N] DOF ids (a + nmax), then perm (a)
};

struct BoxRun {     // device-written results per processed box
  int s, r, n, nq;
};

struct SolveBox;

struct LevelDev {   // device state of a level
  const BoxDesc* desc;
  BoxRun* run;
  const int* nlist;
  const int* qlist;
  const int64_t* pairtab;
  const int64_t* qpair;
  int* cur_n;        // current active count per current box
  const int* cur_off;// offset of a box's act0 in act_dof / act_pos
  const int* cur_a0; // a0 per current box
  const int* act_dof;
  int* act_pos;
  double2* delta;    // Schur-update pool
  int* rows;         // int scratch
  void* Mbuf;        // ID scratch (double2 or float2)
  double2* Wbuf;
  double2* arena;    // factor arena (G1, G3, T, Xinv)
  int* iarena;       // factor int arena (idx)
  int n_proxy;
  double proxy_factor;
  double eps;
  int* status;
  // X_RR^{-1} by fp32 inversion + Newton-Schulz refinement (boxes with
  // kNsMin <= r <= ns_rmax): per box (descriptor index) the offset of its
  // X_RR copy and product scratch (2 a^2 values) and its refinement residual
  double2* nsbuf;
  const int64_t* ns_off;
  unsigned long long* ns_err;   // max |I - X_RR X_1| per box, as double bits
  int ns_rmax;
  const unsigned char* ns_skip = nullptr;   // per box: skip this refinement step
  // root block elimination on the tensor cores (one step: block [i0, i0 + r))
  double2* root_A;   // n0 x n0, ld n0
  double2* root_W;   // later x r, ld later
  int64_t root_n0;
  int root_i0, root_r;
  // C products of the solve sweeps on the tensor cores: the LevelDev of a
  // solve plan, whose desc/run are placeholder arrays indexed like sbox
  const SolveBox* sbox;
  double2* sv;       // permuted right-hand sides, N x nrhs
  int64_t sn;
  int snrhs;
  double2* spart;    // partial-sum area (z and t slots), stride spst per rhs
  int64_t spst;
};
constexpr int kNsMin = 32;      // smallest r refined on the tensor cores

// one per eliminated box, in elimination order (solve plan)
struct SolveBox {
  int r, s, n, zoff;       // zoff: the box's r scratch values (its first chunk's partials)
  int toff;                // r values: the summed partials of the backward sweep
  int item_beg, item_cnt;  // chunks of C = [S | N] (SweepItem list)
  const int* idx;          // [R | S | N]
  const double2* T;  int ldT;
  const double2* Xinv; int ldX;
  const double2* XCR; int ldL;   // (s+n) x r
  const double2* XRC; int ldU;   // r x (s+n)
};

// a chunk [c0, c1) of a box's C rows (forward) or columns (backward)
constexpr int kSweepChunkDefault = 64;
struct SweepItem {
  int box;       // index into the SolveBox array
  int c0, c1;
  int part;      // offset of this chunk's r partial sums (per right-hand side)
};
// one colour of one level in the solve plan
struct SweepSeg {
  int b0, nb;    // boxes [b0, b0 + nb) of the SolveBox array
  int i0, ni;    // C-chunk items [i0, i0 + ni)
  int ri0, nri;  // R-row chunk items
  int si0, nsi;  // S-row chunk items
  int rmax, smax;
  int chunk;     // rows (forward) or columns (backward) of C per item
  int64_t part;  // partial sums needed per right-hand side
  double flops_c, bytes_c;   // per sweep: X_CR / X_RC products (per rhs: flops)
  double flops_b, bytes_b;   // per sweep: T and X_RR^{-1} products
  double bytes_per_rhs;      // vector bytes read and written per right-hand side
};

// ---------------------------------------------------------------------------
// launch accounting: every kernel launch of the library goes through
// FMMLU_LAUNCH, which counts it and, when a profiler is active on the calling
// thread, brackets it with CUDA events on its stream.
// ---------------------------------------------------------------------------
void launch_begin(const char* name, cudaStream_t st);
void launch_end(const char* name, cudaStream_t st);
#define FMMLU_LAUNCH(name, st, ...)          \
  do {                                       \
    ::fmmlu::launch_begin(name, (st));       \
    __VA_ARGS__;                             \
    ::fmmlu::launch_end(name, (st));         \
  } while (0)

// ---------------------------------------------------------------------------
// launch wrappers (defined in the .cu files)
// ---------------------------------------------------------------------------
// tree.cu: see tree_host.h (gpu_build_tree)
// assembly.cu
void launch_permute_geometry(const double* pts, const double* nrm, const double* w,
                             const int* perm, int64_t n, double* soa, cudaStream_t st);
// fills the 10 n floats of `fsoa` from the sorted SoA and returns the views
GeometryF launch_split_geometry(const double* soa, int64_t n, float* fsoa, cudaStream_t st);
void launch_gather_rows(const LevelDev& L, int b0, int nb, cudaStream_t st);
// fp32: kernel values in single precision from g.f (cudaErrorInvalidValue
// when those copies were not made)
cudaError_t launch_assemble_id(const LevelDev& L, const Geometry& g, int b0, int nb,
                               int mmax_max, bool fp32, cudaStream_t st);
cudaError_t launch_assemble_elim(const LevelDev& L, const Geometry& g, int b0, int nb,
                                 int amax, int nmax_max, bool fp32, cudaStream_t st);
struct MergeItem {
  const double2* src; double2* dst;
  int ld_src, ld_dst, off_i, off_j, ni, nj;
  const int* pos_i; const int* pos_j;
};
void launch_merge(const MergeItem* items, int nitems, int max_ni, int max_nj,
                  cudaStream_t st);
void launch_assemble_root(const Geometry& g, const int* dofs, const int* owner,
                          const int* pos, const int64_t* pairoff, const int* a0,
                          int ncur, const double2* delta, int n0, double2* A,
                          cudaStream_t st);
void launch_matvec(const Geometry& g, int64_t n, const double2* v, double2* y,
                   int nrhs, cudaStream_t st);
// linalg.cu
void launch_cpqr(const LevelDev& L, int b0, int nb, bool fp32, int amax,
                 cudaStream_t st);
// cpqr_dist.cu: one box over P cooperating CTAs (cooperative launch)
struct CpqrPart {
  int box;       // descriptor index of the box
  int rank;      // 0 .. P-1
  int P;         // CTAs of this box
  int pad_;
  int64_t scratch_off;   // byte offset of the box's scratch
};
size_t cpqr_dist_scratch_bytes(int P, int a, bool fp32);
int cpqr_dist_capacity(int amax, bool fp32);
cudaError_t launch_cpqr_dist(const LevelDev& L, const CpqrPart* d_parts, int nparts,
                             unsigned char* scratch, int amax, bool fp32, cudaStream_t st);
// ozaki.cu: Schur update on bf16 tensor cores by exact operand splitting
struct OzBoxHost {       // per box of a colour, planned from bounds
  int64_t a_off;         // bf16 offset of W's slices: [p][part][mpad][kp]
  int64_t b_off;         // bf16 offset of X_RC's slices: [q][part][mpad][kp]
  int64_t e_off;         // int offset of row exponents (mpad) then column exponents (mpad)
  int mpad, kp;          // rows/cols padded to 64, k padded to 16
};
void plan_oz_box(int a, int nmax, int64_t& slice_off, int64_t& expo_off, OzBoxHost& out);
void launch_oz_schur(const LevelDev& L, int b0, int nb, const OzBoxHost* d_oz, void* slices,
                     int* expo, int amax, int nmax_max, cudaStream_t st);
// which: 0 = G1 update, 1 = G3 update, 2 = W = X_CR X_RR^{-1}
void launch_oz_elim_gemms(const LevelDev& L, int b0, int nb, const OzBoxHost* d_oz, void* slices,
                          int* expo, int amax, int nmax_max, int which, cudaStream_t st);
constexpr int kOzInnerMin = 32;   // inner dimension from which the mma.sync path is used
constexpr int kTcInnerMin = 1;    // inner dimension from which the tcgen05 path is used
// Gram form of the ID (ozaki.cu, pchol.cu): G = M^H M of the ID matrix on the
// tensor cores, then greedy pivoted Cholesky of G -- the same column selection
// and the same R (up to row phases) as CPQR of M in exact arithmetic.
struct GramBoxHost {     // per box of a level, planned from bounds
  int64_t sl_off;        // bf16 offset of M's column slices: [p][part][apad][kp]
  int64_t e_off;         // int offset of the apad column exponents
  int64_t G_off;         // double2 offset of G (a x a), then R by columns (a x a)
  int apad, kp;          // a padded to 64; mmax padded to 16
};
void plan_gram_box(int a, int mmax, bool fp32, int64_t& slice_off, int64_t& expo_off,
                   int64_t& g_off, GramBoxHost& out);
void launch_gram(const LevelDev& L, int b0, int nb, const GramBoxHost* d_gb, void* slices,
                 int* expo, double2* gbuf, int amax, int mmax, bool fp32, cudaStream_t st);
size_t pchol_scratch_bytes(int P);
size_t pchol_smem(int amax);   // dynamic shared memory of one CTA
int pchol_capacity(int amax);
cudaError_t launch_pchol(const LevelDev& L, const CpqrPart* d_parts, int nparts,
                         unsigned char* scratch, const GramBoxHost* d_gb, double2* gbuf, int amax,
                         bool cooperative, cudaStream_t st);
// tcgemm.cu: exact-split complex products on tcgen05 tensor cores (TMEM
// accumulators, bulk-copy operand pipeline)
struct TcBoxHost {       // per box of a colour, planned from bounds
  int64_t a_off, b_off;  // byte offsets of the A and B digit slices
  int64_t ea_off, eb_off;  // int offsets of the row / column exponents
};
void plan_tc_box(int mrows, int ncols, int k, int ns, int64_t& slice_off, int64_t& expo_off,
                 TcBoxHost& out);
size_t tc_smem_bytes(int ns);
// problems of the tcgen05 path
enum { kTcG1 = 0, kTcG3 = 1, kTcW = 2, kTcSchur = 3, kTcXrr = 4, kTcGram = 5, kTcNsY = 6,
       kTcNsX = 7, kTcRootW = 8, kTcRootS = 9,
       // solve sweeps: b_C -= op(X_CR) z (forward) and t = op(X_RC) x_C
       // (backward), op = identity or, for the adjoint (suffix A), the
       // conjugate transpose of the other block
       kTcSvC = 10, kTcSvT = 11, kTcSvCA = 12, kTcSvTA = 13 };
struct TcUnit {          // one CTA of a tcgen05-path launch
  int box;               // box index relative to the colour's first box
  int side;              // 0 = A operand, 1 = B operand (split launches); product
                         // units of a split-K problem: k16 steps per chunk
  int x, y;              // row block and k group (split) or tile (product)
};
struct TcBoxSize {       // exact (or bounding) sizes of one box on the host
  int a, s, r, n, kgram;
  int nsmax;             // largest r refined by Newton-Schulz
  int nrhs;              // right-hand sides (solve products)
};
struct TcPlan {          // the five launches of one problem: offsets into the unit list
  int off[5], cnt[5];    // exponents A, B; digits A, B; product tiles
};
// gram_chunk: k16 steps per split-K chunk of the Gram product (kTcGram only;
// every chunk length gives the same exact sums)
constexpr int kGramChunkDefault = 128;
void tc_plan(int which, const std::vector<TcBoxSize>& boxes, std::vector<TcUnit>& units,
             TcPlan& plan, int gram_chunk = kGramChunkDefault);
void launch_tc_planned(int which, const LevelDev& L, int b0, const TcBoxHost* d_tb, void* slices,
                       int* expo, const GramBoxHost* d_gb, double2* gbuf, bool fp32,
                       const TcUnit* d_units, const TcPlan& pl, cudaStream_t st,
                       unsigned long long* gx = nullptr, const int64_t* gx_off = nullptr);
// G of a colour's boxes (units: one per box) from the Gram product's split-K
// int64 accumulator
void launch_gram_finalize(const LevelDev& L, int b0, const TcUnit* d_boxes, int nboxes, int amax,
                          const TcBoxHost* d_tb, const int* expo, const GramBoxHost* d_gb,
                          double2* gbuf, unsigned long long* gx, const int64_t* gx_off, bool fp32,
                          cudaStream_t st);
// gj_dist.cu: fp32 Gauss-Jordan of X_RR over a thread-block cluster per box
// (units: one per box, TcUnit::box relative to b0); writes the fp32 inverse to
// Xinv (as complex128) and a complex128 copy of X_RR to nsbuf
size_t gj32_smem(int rmax, int P);
int gj32_cluster_size(int rmax);                 // 0: no cluster shape fits
cudaError_t launch_gj32(const LevelDev& L, int b0, const TcUnit* d_units, int nunits, int rmax,
                        int P, cudaStream_t st);
// linalg.cu: boxes of the refinement whose residual exceeds `thr` are
// inverted again in fp64 from the stored copy of X_RR (one CTA per box)
void launch_ns_fallback(const LevelDev& L, int b0, const TcUnit* d_units, int nunits, int amax,
                        double thr, cudaStream_t st);
// flags the refined boxes whose first residual e already bounds the next
// iterate's by (r e)^2 <= thr, so that a third step can skip them (skip[b]
// = 1), and clears their residual record
void launch_ns_flag(const LevelDev& L, int b0, const TcUnit* d_units, int nunits, double thr,
                    unsigned char* skip, cudaStream_t st);
// gj_dist.cu: X_RR^{-1} of one box over P cooperating CTAs (cooperative launch)
size_t gj_dist_scratch_bytes(int a);
int gj_dist_capacity(int amax);
cudaError_t launch_gj_dist(const LevelDev& L, const CpqrPart* d_parts, int nparts,
                           unsigned char* scratch, int amax, cudaStream_t st);
// kskip > 0: leave boxes whose inner dimension is >= kskip to the tensor-core path
void launch_gemm_g1(const LevelDev& L, int b0, int nb, int amax, int nmax_max,
                    cudaStream_t st, int kskip = 0);
void launch_gemm_g3(const LevelDev& L, int b0, int nb, int amax, int nmax_max,
                    cudaStream_t st, int kskip = 0);
void launch_gemm_xrr(const LevelDev& L, int b0, int nb, int amax, cudaStream_t st, int kskip = 0);
void launch_xrr_inverse(const LevelDev& L, int b0, int nb, int amax, cudaStream_t st,
                        int skip_lo = 1, int skip_hi = 0);
void launch_gemm_w(const LevelDev& L, int b0, int nb, int amax, int nmax_max,
                   cudaStream_t st, int kskip = 0);
void launch_schur_update(const LevelDev& L, int b0, int nb, int amax, int nmax_max,
                         cudaStream_t st, int kskip = 0);
cudaError_t launch_root_factor(double2* A, int n0, int nb, double2* work, int* status,
                               cudaStream_t st, bool tensor_cores = false);
void launch_root_diag(double2* A, int n0, int i0, int r, int* status, cudaStream_t st);
cudaError_t launch_root_factor_tc(double2* A, int n0, int nb, double2* W, int* status,
                                  cudaStream_t st);
// solve.cu
void launch_gather_vec(const double2* b, const int* perm, int64_t n, int nrhs,
                       double2* v, cudaStream_t st);
void launch_scatter_vec(const double2* v, const int* perm, int64_t n, int nrhs,
                        double2* x, cudaStream_t st);
// one-time kernel attributes of the sweeps (call before a stream capture)
void prepare_solve_kernels();
// cnt: one int per eliminated box and right-hand side, zero between sweeps.
// skip_c: leave out the C product (k_fwd_c / k_bwd_t) because the caller
// runs it on the tensor cores (forward: then launch_copy_z stores b_R = z)
void launch_sweep(const SolveBox* boxes, const SweepItem* items, const SweepSeg& sg,
                  double2* v, int64_t n, int nrhs, bool backward, bool adjoint,
                  double2* partial, int64_t pstride, cudaStream_t st, int* cnt,
                  bool skip_c = false);
// b_R = z for the boxes [b0, b0 + nb) (z in the boxes' z slots)
void launch_copy_z(const SolveBox* boxes, int b0, int nb, int rmax, double2* v, int64_t n,
                   int nrhs, const double2* partial, int64_t pstride, cudaStream_t st);
void launch_root_gather(const double2* v, const int* dofs, int n0, int64_t n,
                        int nrhs, double2* vr, cudaStream_t st);
void launch_root_scatter(const double2* vr, const int* dofs, int n0, int64_t n,
                         int nrhs, double2* v, cudaStream_t st);
// scratch: root_solve_scratch_bytes(n0, nb, nrhs) bytes of device memory
size_t root_solve_scratch_bytes(int n0, int nb, int nrhs);
cudaError_t launch_root_solve(const double2* A, int n0, int nb, double2* vr, double2* z,
                              void* scratch, int nrhs, bool adjoint, cudaStream_t st);
// sonar.cu (plane waves and the backscattered far field, caller order)
int backscatter_blocks(int64_t n);   // partial sums per direction
void launch_plane_waves(const double* pts, const double* w, int64_t n, double k,
                        const double* dirs, int m0, int mcount, double2* b, cudaStream_t st);
void launch_backscatter(const double* pts, const double* nrm, const double* w, int64_t n,
                        double k, double eta, const double* dirs, int m0, int mcount,
                        const double2* x, double2* part, double2* R, cudaStream_t st);
// krylov.cu (preconditioned GMRES: basis of at most kKrMaxRestart + 1 vectors)
constexpr int kKrMaxRestart = 64;
constexpr int kKrMaxBasis = kKrMaxRestart + 1;
int kr_blocks(int64_t n);   // partial sums per inner product (size of `part` / ncols)
void launch_kr_dots(const double2* V, int64_t ldv, int ncols, const double2* w, int64_t n,
                    double2* part, double2* hc, double2* hacc, cudaStream_t st);
void launch_kr_update(double2* w, const double2* V, int64_t ldv, int ncols, const double2* hc,
                      int64_t n, cudaStream_t st);
void launch_kr_scale(double2* dst, const double2* src, const double* scal, int64_t n,
                     cudaStream_t st);
void launch_kr_residual(double2* r, const double2* b, const double2* y, int64_t n,
                        cudaStream_t st);
void launch_kr_add(double2* x, const double2* z, int64_t n, cudaStream_t st);
void launch_kr_combine(double2* u, const double2* V, int64_t ldv, int ncols, const double2* y,
                       int64_t n, cudaStream_t st);
void launch_kr_givens(double2* H, int ldh, int j, const double2* nrm2, double* cs, double2* sn,
                      double2* g, double* scal, double* est, cudaStream_t st);
void launch_kr_start(const double2* nrm2, double2* g, int len, double* scal, double* est,
                     cudaStream_t st);
void launch_kr_trisolve(const double2* H, int ldh, int jd, const double2* g, double2* y,
                        cudaStream_t st);

}  // namespace fmmlu
