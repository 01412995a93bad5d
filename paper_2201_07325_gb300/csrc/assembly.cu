// Assembly kernels: every matrix entry the factorization reads is generated
// here from the kernel (device_common.cuh) plus the stored Schur updates.
//
//  * k_gather_rows   -- current active DOFs of Q(B) and N(B) (Sec. 4.2: only
//                       active DOFs of a region take part).
//  * k_assemble_id   -- the stacked matrix of the simultaneous skeletonization
//                       (Sec. 5.1)   [ A_QB ; A_BQ^T ; c K_gB sqrt(D_B) ;
//                                      c S_Bg^T sqrt(D_B) ],
//                       c = sqrt(4 pi rho^2 / n_gamma), proxy points on a
//                       sphere of radius rho around B's centre.
//  * k_assemble_elim -- the blocks of Eq. strong-skel-elim in pivoted order:
//                       G1 = A[B_piv, (S|N|R)] and G3 = A[(S|N|R), B_piv].
//  * k_merge         -- level change: the Schur blocks of children restricted to
//                       their skeletons become blocks of the parents (Sec. 4.2,
//                       actives of a parent = union of its children's skeletons).
//  * k_assemble_root -- the remaining dense block A_{B_t B_t}.
//  * k_matvec        -- dense on-the-fly A v (independent of the factorization).
#include "device_common.cuh"
#include "dfloat.cuh"

namespace fmmlu {

__global__ void k_permute_geometry(const double* __restrict__ pts, const double* __restrict__ nrm,
                                   const double* __restrict__ w, const int* __restrict__ perm,
                                   int64_t n, double* soa) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t p = perm[i];
  soa[0 * n + i] = pts[3 * p + 0];
  soa[1 * n + i] = pts[3 * p + 1];
  soa[2 * n + i] = pts[3 * p + 2];
  soa[3 * n + i] = nrm[3 * p + 0];
  soa[4 * n + i] = nrm[3 * p + 1];
  soa[5 * n + i] = nrm[3 * p + 2];
  soa[6 * n + i] = w[p];
  soa[7 * n + i] = sqrt(w[p]);
}

void launch_permute_geometry(const double* pts, const double* nrm, const double* w,
                             const int* perm, int64_t n, double* soa, cudaStream_t st) {
  FMMLU_LAUNCH("permute_geometry", st,
               k_permute_geometry<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pts, nrm, w, perm, n, soa));
}

__global__ void k_split_geometry(const double* __restrict__ soa, int64_t n, float* __restrict__ f) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int c = 0; c < 3; ++c) {
    const double x = soa[c * n + i];
    const float h = (float)x;
    f[c * n + i] = h;
    f[(3 + c) * n + i] = (float)(x - (double)h);
    f[(6 + c) * n + i] = (float)soa[(3 + c) * n + i];
  }
  f[9 * n + i] = (float)soa[7 * n + i];
}

GeometryF launch_split_geometry(const double* soa, int64_t n, float* f, cudaStream_t st) {
  if (n > 0)
    FMMLU_LAUNCH("split_geometry", st,
                 k_split_geometry<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(soa, n, f));
  return GeometryF{f, f + n, f + 2 * n, f + 3 * n, f + 4 * n, f + 5 * n,
                   f + 6 * n, f + 7 * n, f + 8 * n, f + 9 * n};
}

// ---------------------------------------------------------------------------

__global__ void k_gather_rows(LevelDev L, int b0) {
  int b = b0 + blockIdx.x;
  const BoxDesc d = L.desc[b];
  int* qdof = L.rows + d.rows_off;
  int* qpos = qdof + d.qmax;
  int* qloc = qpos + d.qmax;
  int* ndof = qloc + d.qmax;
  int* npos = ndof + d.nmax;
  int* nloc = npos + d.nmax;
  int off = 0;
  for (int c = 0; c < d.qcnt; ++c) {
    int C = L.qlist[d.qbeg + c];
    int nC = L.cur_n[C];
    int base = L.cur_off[C];
    for (int i = threadIdx.x; i < nC; i += blockDim.x) {
      int p = L.act_pos[base + i];
      qdof[off + i] = L.act_dof[base + p];
      qpos[off + i] = p;
      qloc[off + i] = c;
    }
    off += nC;
  }
  int nq = off;
  off = 0;
  for (int c = 0; c < d.ncnt; ++c) {
    int C = L.nlist[d.nbeg + c];
    int nC = L.cur_n[C];
    int base = L.cur_off[C];
    for (int i = threadIdx.x; i < nC; i += blockDim.x) {
      int p = L.act_pos[base + i];
      ndof[off + i] = L.act_dof[base + p];
      npos[off + i] = p;
      nloc[off + i] = c + 1;
    }
    off += nC;
  }
  if (threadIdx.x == 0) {
    L.run[b].nq = nq;
    L.run[b].n = off;
    if (nq > d.qmax || off > d.nmax) set_status(L.status, kStatusBound);
  }
}

void launch_gather_rows(const LevelDev& L, int b0, int nb, cudaStream_t st) {
  if (nb <= 0) return;
  FMMLU_LAUNCH("gather_rows", st, k_gather_rows<<<nb, 256, 0, st>>>(L, b0));
}

// ---------------------------------------------------------------------------

constexpr int kIdRows = 64;   // most half-rows per block (pairs of rows)

// The rows come in pairs that share a kernel evaluation: row i < nq (A(q_i, b_j),
// outgoing ring) and row nq + i (A(b_j, q_i), incoming ring, the transpose
// block); proxy row 2nq + l (K(y_l, b_j)) and 2nq + np + l (G(b_j, y_l)).
// A block takes `rpb` row pairs of one box; the proxy points of its rows are
// computed once, before the entries. In single precision (C = float2) the
// kernel is evaluated from the split fp32 geometry and the Schur updates are
// added in fp32; in double precision everything is fp64.
// a Schur update added to an ID-matrix entry: complex64 entries take it
// narrowed from its bit pattern (the high and low fp32 parts, summed)
__device__ __forceinline__ double2 id_delta(double2 v, double2) { return v; }
__device__ __forceinline__ float2 id_delta(double2 v, float2) {
  const DF x = df_split_bits(v.x), y = df_split_bits(v.y);
  return make_float2(x.h + x.l, y.h + y.l);
}

template <typename C>
__global__ void k_assemble_id(LevelDev L, Geometry g, int b0, int rpb) {
  using R = decltype(C().x);
  constexpr bool kF = sizeof(R) == 4;
  __shared__ double s_yd[kIdRows][3];   // rho u_l of the block's proxy rows
  __shared__ float s_yf[kIdRows][3];
  int b = b0 + blockIdx.y;
  const BoxDesc d = L.desc[b];
  const int nq = L.run[b].nq;
  const int np = L.n_proxy;
  const int half = nq + np;
  const int row0 = blockIdx.x * rpb;
  if (row0 >= half) return;
  const int a = d.a;
  const int* qdof = L.rows + d.rows_off;
  const int* qpos = qdof + d.qmax;
  const int* qloc = qpos + d.qmax;
  const int bbase = L.cur_off[d.cur];
  C* M = reinterpret_cast<C*>(L.Mbuf) + d.M_off;
  const double rho = L.proxy_factor * 0.86602540378443864676 * d.h;
  const double cg = sqrt(4.0 * kPi * rho * rho / np);
  const int rows = min(rpb, half - row0);
  for (int t = threadIdx.x; t < rows; t += blockDim.x) {
    const int l = row0 + t - nq;
    if (l >= 0) {
      double ux, uy, uz;
      fib_point(l, np, ux, uy, uz);
      s_yd[t][0] = rho * ux; s_yd[t][1] = rho * uy; s_yd[t][2] = rho * uz;
      s_yf[t][0] = (float)s_yd[t][0]; s_yf[t][1] = (float)s_yd[t][1];
      s_yf[t][2] = (float)s_yd[t][2];
    }
  }
  __syncthreads();
  const R kk = (R)g.k, ee = (R)g.eta;
  // the box centre split like the points (single precision)
  const float chx = (float)d.cx, chy = (float)d.cy, chz = (float)d.cz;
  const float clx = (float)(d.cx - (double)chx), cly = (float)(d.cy - (double)chy),
              clz = (float)(d.cz - (double)chz);
  const R cgr = (R)cg;
  for (int e = threadIdx.x; e < rows * a; e += blockDim.x) {
    const int t = e % rows;
    const int i = row0 + t;
    const int j = e / rows;
    const int jd = L.act_dof[bbase + j];
    C v_out, v_in;
    int r_out, r_in;
    if (i < nq) {
      const int q = qdof[i];
      C kqb, kbq, gq;
      R sc;
      if constexpr (kF) {
        const GeometryF& f = g.f;
        comb_kernel_pair<float>(fdiff(f.xh, f.xl, jd, q), fdiff(f.yh, f.yl, jd, q),
                                fdiff(f.zh, f.zl, jd, q), f.nx[q], f.ny[q], f.nz[q], f.nx[jd],
                                f.ny[jd], f.nz[jd], kk, ee, kqb, kbq, gq);
        sc = f.sw[q] * f.sw[jd];
      } else {
        comb_kernel_pair<double>(g.px[jd] - g.px[q], g.py[jd] - g.py[q], g.pz[jd] - g.pz[q],
                                 g.nx[q], g.ny[q], g.nz[q], g.nx[jd], g.ny[jd], g.nz[jd], kk, ee,
                                 kqb, kbq, gq);
        sc = g.sw[q] * g.sw[jd];
      }
      C o = cscale(kqb, sc), tr = cscale(kbq, sc);
      const int64_t off_o = L.qpair[d.qpair + 2 * qloc[i]];
      if (off_o >= 0) {
        const int ldc = L.cur_a0[L.qlist[d.qbeg + qloc[i]]];
        o = cadd(o, id_delta(L.delta[off_o + qpos[i] + (int64_t)j * ldc], C()));
      }
      const int64_t off_i = L.qpair[d.qpair + 2 * qloc[i] + 1];
      if (off_i >= 0) tr = cadd(tr, id_delta(L.delta[off_i + j + (int64_t)qpos[i] * a], C()));
      v_out = o;
      v_in = tr;
      r_out = i;
      r_in = nq + i;
    } else {
      const int l = i - nq;
      C kyb, kby, gy;
      R sc;
      if constexpr (kF) {
        const GeometryF& f = g.f;
        const float rx = (f.xh[jd] - chx) + (f.xl[jd] - clx);   // b_j - centre
        const float ry = (f.yh[jd] - chy) + (f.yl[jd] - cly);
        const float rz = (f.zh[jd] - chz) + (f.zl[jd] - clz);
        comb_kernel_pair<float>(rx - s_yf[t][0], ry - s_yf[t][1], rz - s_yf[t][2], 0.f, 0.f, 0.f,
                                f.nx[jd], f.ny[jd], f.nz[jd], kk, ee, kyb, kby, gy);
        sc = cgr * f.sw[jd];
      } else {
        const double yx = d.cx + s_yd[t][0], yy = d.cy + s_yd[t][1], yz = d.cz + s_yd[t][2];
        comb_kernel_pair<double>(g.px[jd] - yx, g.py[jd] - yy, g.pz[jd] - yz, 0.0, 0.0, 0.0,
                                 g.nx[jd], g.ny[jd], g.nz[jd], kk, ee, kyb, kby, gy);
        sc = cg * g.sw[jd];
      }
      v_out = cscale(kyb, sc);   // K(y_l, b_j): outgoing proxy row
      v_in = cscale(gy, sc);     // G(b_j, y_l): incoming proxy row
      r_out = 2 * nq + l;
      r_in = 2 * nq + np + l;
    }
    M[r_out + (int64_t)j * d.mmax] = v_out;
    M[r_in + (int64_t)j * d.mmax] = v_in;
  }
}

cudaError_t launch_assemble_id(const LevelDev& L, const Geometry& g, int b0, int nb, int mmax_max,
                               bool fp32, cudaStream_t st) {
  if (nb <= 0) return cudaSuccess;
  if (fp32 && !g.f.xh) return cudaErrorInvalidValue;   // single-precision copies not made
  // m = 2 (nq + np) rows, in pairs. Every entry is computed the same way for
  // any blocking, so colours with few boxes get shorter row blocks: the
  // kernel is fp64-bound per SM and needs every SM busy.
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 148;
  }
  const int half = mmax_max / 2;
  int rpb = kIdRows;
  while (rpb > 8 && (int64_t)((half + rpb - 1) / rpb) * nb < 4 * (int64_t)sms) rpb >>= 1;
  dim3 grid((half + rpb - 1) / rpb, nb);
  if (fp32)
    FMMLU_LAUNCH("assemble_id", st, k_assemble_id<float2><<<grid, 256, 0, st>>>(L, g, b0, rpb));
  else
    FMMLU_LAUNCH("assemble_id", st, k_assemble_id<double2><<<grid, 256, 0, st>>>(L, g, b0, rpb));
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// elimination blocks in pivoted order

struct Idx {
  int dof, loc, pos;
};

__device__ __forceinline__ Idx bpiv(const LevelDev& L, const BoxDesc& d, const int* perm, int i) {
  int p = perm[i];
  return Idx{L.act_dof[L.cur_off[d.cur] + p], 0, p};
}

// G1 = A[B_piv, (S|N|R)] (a x (a+n), ld a) and G3 = A[(S|N|R), B_piv]
// ((a+n) x a, ld a+nmax): G3[j][i] is the transposed pair of G1[i][j], so one
// kernel evaluation gives both. A block takes 32 x 32 pairs (i in B_piv, j in
// [S|N|R]); G1 is written along i, G3 through a shared-memory transpose along j.
constexpr int kElimT = 32;

__device__ __forceinline__ Idx col_idx(const LevelDev& L, const BoxDesc& d, const int* perm,
                                       const int* ndof, const int* npos, const int* nloc, int s,
                                       int n, int j) {
  return j < s ? bpiv(L, d, perm, j)
               : (j < s + n ? Idx{ndof[j - s], nloc[j - s], npos[j - s]} : bpiv(L, d, perm, j - n));
}

__device__ __forceinline__ double2 add_delta(const LevelDev& L, const BoxDesc& d, double2 v, Idx r,
                                             Idx c) {
  const int cnt = 1 + d.ncnt;
  const int64_t off = L.pairtab[d.pairtab + (int64_t)r.loc * cnt + c.loc];
  if (off >= 0) {
    const int ld = r.loc == 0 ? d.a : L.cur_a0[L.nlist[d.nbeg + r.loc - 1]];
    v = cadd(v, L.delta[off + r.pos + (int64_t)c.pos * ld]);
  }
  return v;
}

// kF: off-diagonal kernel values in fp32 from the split geometry (the mixed
// path), converted to fp64 before the Schur updates are added; the diagonal
// (self) entries are always fp64.
template <bool kF>
__global__ void __launch_bounds__(256) k_assemble_elim(LevelDev L, Geometry g, int b0) {
  __shared__ double2 t3[kElimT][kElimT + 1];
  const int b = b0 + blockIdx.y;
  const BoxDesc d = L.desc[b];
  const BoxRun run = L.run[b];
  const int a = d.a, s = run.s, n = run.n;
  if (s >= a) return;   // nothing to eliminate
  const int ti = (a + kElimT - 1) / kElimT, tj = (a + n + kElimT - 1) / kElimT;
  if ((int)blockIdx.x >= ti * tj) return;
  const int i0 = (blockIdx.x % ti) * kElimT, j0 = (blockIdx.x / ti) * kElimT;
  const int* perm = L.iarena + d.idx_off + d.a + d.nmax;
  const int* ndof = L.rows + d.rows_off + 3 * d.qmax;
  const int* npos = ndof + d.nmax;
  const int* nloc = npos + d.nmax;
  double2* G1 = L.arena + d.G1_off;
  double2* G3 = L.arena + d.G3_off;
  const int ld3 = a + d.nmax;
  const int li = threadIdx.x & 31;
  const float kf = (float)g.k, ef = (float)g.eta;
  for (int lj = threadIdx.x >> 5; lj < kElimT; lj += blockDim.x >> 5) {
    const int i = i0 + li, j = j0 + lj;
    if (i < a && j < a + n) {
      const Idx r = bpiv(L, d, perm, i);
      const Idx c = col_idx(L, d, perm, ndof, npos, nloc, s, n, j);
      double2 arc, acr;
      if (kF && r.dof != c.dof) {
        float2 fa, fb;
        entry_pair_f(g.f, kf, ef, r.dof, c.dof, fa, fb);
        // widened from the bit patterns: the conversion instruction would
        // occupy GB300's narrow fp64 pipe
        arc = make_double2(f2d_bits(fa.x), f2d_bits(fa.y));
        acr = make_double2(f2d_bits(fb.x), f2d_bits(fb.y));
      } else {
        entry_pair(g, r.dof, c.dof, arc, acr);
      }
      G1[i + (int64_t)j * a] = add_delta(L, d, arc, r, c);
      t3[lj][li] = add_delta(L, d, acr, c, r);
    }
  }
  __syncthreads();
  const int lj = threadIdx.x & 31;
  for (int lii = threadIdx.x >> 5; lii < kElimT; lii += blockDim.x >> 5) {
    const int i = i0 + lii, j = j0 + lj;
    if (i < a && j < a + n) G3[j + (int64_t)i * ld3] = t3[lj][lii];
  }
}

cudaError_t launch_assemble_elim(const LevelDev& L, const Geometry& g, int b0, int nb, int amax,
                                 int nmax_max, bool fp32, cudaStream_t st) {
  if (nb <= 0) return cudaSuccess;
  if (fp32 && !g.f.xh) return cudaErrorInvalidValue;   // single-precision copies not made
  const int ti = (amax + kElimT - 1) / kElimT, tj = (amax + nmax_max + kElimT - 1) / kElimT;
  dim3 grid((unsigned)(ti * tj), nb);
  if (fp32)
    FMMLU_LAUNCH("assemble_elim", st, k_assemble_elim<true><<<grid, 256, 0, st>>>(L, g, b0));
  else
    FMMLU_LAUNCH("assemble_elim", st, k_assemble_elim<false><<<grid, 256, 0, st>>>(L, g, b0));
  return cudaSuccess;
}

// ---------------------------------------------------------------------------

__global__ void k_merge(const MergeItem* __restrict__ items) {
  const MergeItem it = items[blockIdx.x];
  int64_t tot = (int64_t)it.ni * it.nj;
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    int i = (int)(e % it.ni), j = (int)(e / it.ni);
    double2 v = it.src[it.pos_i[i] + (int64_t)it.pos_j[j] * it.ld_src];
    it.dst[(it.off_i + i) + (int64_t)(it.off_j + j) * it.ld_dst] = v;
  }
}

void launch_merge(const MergeItem* items, int nitems, int, int, cudaStream_t st) {
  if (nitems <= 0) return;
  FMMLU_LAUNCH("merge", st, k_merge<<<nitems, 256, 0, st>>>(items));
}

// ---------------------------------------------------------------------------

__global__ void k_assemble_root(Geometry g, const int* __restrict__ dofs,
                                const int* __restrict__ owner, const int* __restrict__ pos,
                                const int64_t* __restrict__ pairoff, const int* __restrict__ a0,
                                int ncur, const double2* __restrict__ delta, int n0,
                                double2* A) {
  int i = blockIdx.x * 32 + threadIdx.x;
  int j0 = blockIdx.y * 32;
  if (i >= n0) return;
  int oi = owner[i], pi = pos[i], di = dofs[i];
  for (int jj = threadIdx.y; jj < 32; jj += blockDim.y) {
    int j = j0 + jj;
    if (j >= n0) break;
    int oj = owner[j];
    double2 v = entry(g, di, dofs[j]);
    int64_t off = pairoff[(int64_t)oi * ncur + oj];
    if (off >= 0) v = cadd(v, delta[off + pi + (int64_t)pos[j] * a0[oi]]);
    A[i + (int64_t)j * n0] = v;
  }
}

void launch_assemble_root(const Geometry& g, const int* dofs, const int* owner, const int* pos,
                          const int64_t* pairoff, const int* a0, int ncur,
                          const double2* delta, int n0, double2* A, cudaStream_t st) {
  if (n0 <= 0) return;
  dim3 grid((n0 + 31) / 32, (n0 + 31) / 32);
  FMMLU_LAUNCH("assemble_root", st, k_assemble_root<<<grid, dim3(32, 8), 0, st>>>(
                                         g, dofs, owner, pos, pairoff, a0, ncur, delta, n0, A));
}

// ---------------------------------------------------------------------------

constexpr int kMvTile = 128;

__global__ void k_matvec(Geometry g, int64_t n, const double2* __restrict__ v,
                         double2* __restrict__ y) {
  __shared__ double sx[kMvTile], sy[kMvTile], sz[kMvTile], snx[kMvTile], sny[kMvTile],
      snz[kMvTile], ssw[kMvTile];
  __shared__ double2 sv[kMvTile];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  const double2* vc = v + c * n;
  double tx = 0, ty = 0, tz = 0, tsw = 0;
  if (i < n) { tx = g.px[i]; ty = g.py[i]; tz = g.pz[i]; tsw = g.sw[i]; }
  double2 acc = mk(0.0, 0.0);
  for (int64_t j0 = 0; j0 < n; j0 += kMvTile) {
    __syncthreads();
    for (int t = threadIdx.x; t < kMvTile; t += blockDim.x) {
      int64_t j = j0 + t;
      if (j < n) {
        sx[t] = g.px[j]; sy[t] = g.py[j]; sz[t] = g.pz[j];
        snx[t] = g.nx[j]; sny[t] = g.ny[j]; snz[t] = g.nz[j];
        ssw[t] = g.sw[j]; sv[t] = vc[j];
      }
    }
    __syncthreads();
    if (i < n) {
      int lim = (int)(n - j0 < kMvTile ? n - j0 : kMvTile);
      for (int t = 0; t < lim; ++t) {
        int64_t j = j0 + t;
        double2 aij;
        if (j == i) {
          double w = g.w[i];
          aij = mk(0.5 + g.eta * g.k * w / (4.0 * kPi), -g.eta * sqrt(w / kPi) * 0.5);
        } else {
          aij = cscale(comb_kernel(tx, ty, tz, sx[t], sy[t], sz[t], snx[t], sny[t], snz[t], g.k,
                                   g.eta),
                       tsw * ssw[t]);
        }
        cfma(acc, aij, sv[t]);
      }
    }
  }
  if (i < n) y[c * n + i] = acc;
}

void launch_matvec(const Geometry& g, int64_t n, const double2* v, double2* y, int nrhs,
                   cudaStream_t st) {
  dim3 grid((unsigned)((n + 127) / 128), nrhs);
  FMMLU_LAUNCH("matvec", st, k_matvec<<<grid, 128, 0, st>>>(g, n, v, y));
}

}  // namespace fmmlu
