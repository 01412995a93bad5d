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

constexpr int kIdRows = 64;

template <typename C>
__global__ void k_assemble_id(LevelDev L, Geometry g, int b0) {
  int b = b0 + blockIdx.y;
  const BoxDesc d = L.desc[b];
  int nq = L.run[b].nq;
  int np = L.n_proxy;
  int m = 2 * nq + 2 * np;
  int row0 = blockIdx.x * kIdRows;
  if (row0 >= m) return;
  int a = d.a;
  const int* qdof = L.rows + d.rows_off;
  const int* qpos = qdof + d.qmax;
  const int* qloc = qpos + d.qmax;
  const int bbase = L.cur_off[d.cur];
  C* M = reinterpret_cast<C*>(L.Mbuf) + d.M_off;
  double rho = L.proxy_factor * 0.86602540378443864676 * d.h;
  double cg = sqrt(4.0 * kPi * rho * rho / np);
  int rows = min(kIdRows, m - row0);
  for (int e = threadIdx.x; e < rows * a; e += blockDim.x) {
    int i = row0 + e % rows;
    int j = e / rows;
    int jd = L.act_dof[bbase + j];
    if (sizeof(C) == sizeof(float2)) {
      // mixed path: complex64 kernel blocks (Schur updates rounded to fp32)
      float2 v;
      const float kf = (float)g.k, ef = (float)g.eta;
      if (i < 2 * nq) {
        const bool out = i < nq;
        const int i2 = out ? i : i - nq;
        const int q = qdof[i2];
        const int t = out ? q : jd, sdof = out ? jd : q;
        v = comb_kernel_f(g.px[t], g.py[t], g.pz[t], g.px[sdof], g.py[sdof], g.pz[sdof],
                          (float)g.nx[sdof], (float)g.ny[sdof], (float)g.nz[sdof], kf, ef);
        v = cscale(v, (float)(g.sw[q] * g.sw[jd]));
        int64_t off = L.qpair[d.qpair + 2 * qloc[i2] + (out ? 0 : 1)];
        if (off >= 0) {
          double2 dv = out ? L.delta[off + qpos[i2] + (int64_t)j * L.cur_a0[L.qlist[d.qbeg + qloc[i2]]]]
                           : L.delta[off + j + (int64_t)qpos[i2] * a];
          v = cadd(v, make_float2((float)dv.x, (float)dv.y));
        }
      } else {
        int l = i - 2 * nq;
        bool incoming = l >= np;
        if (incoming) l -= np;
        double ux, uy, uz;
        fib_point(l, np, ux, uy, uz);
        double yx = d.cx + rho * ux, yy = d.cy + rho * uy, yz = d.cz + rho * uz;
        if (!incoming)
          v = comb_kernel_f(yx, yy, yz, g.px[jd], g.py[jd], g.pz[jd], (float)g.nx[jd],
                            (float)g.ny[jd], (float)g.nz[jd], kf, ef);
        else
          v = green_f(g.px[jd], g.py[jd], g.pz[jd], yx, yy, yz, kf);
        v = cscale(v, (float)(cg * g.sw[jd]));
      }
      reinterpret_cast<float2*>(M)[i + (int64_t)j * d.mmax] = v;
      continue;
    }
    double2 v;
    if (i < nq) {
      int q = qdof[i];
      v = entry(g, q, jd);
      int64_t off = L.qpair[d.qpair + 2 * qloc[i]];
      if (off >= 0) {
        int ldc = L.cur_a0[L.qlist[d.qbeg + qloc[i]]];
        v = cadd(v, L.delta[off + qpos[i] + (int64_t)j * ldc]);
      }
    } else if (i < 2 * nq) {
      int i2 = i - nq;
      int q = qdof[i2];
      v = entry(g, jd, q);
      int64_t off = L.qpair[d.qpair + 2 * qloc[i2] + 1];
      if (off >= 0) v = cadd(v, L.delta[off + j + (int64_t)qpos[i2] * a]);
    } else {
      int l = i - 2 * nq;
      bool incoming = l >= np;
      if (incoming) l -= np;
      double ux, uy, uz;
      fib_point(l, np, ux, uy, uz);
      double yx = d.cx + rho * ux, yy = d.cy + rho * uy, yz = d.cz + rho * uz;
      double s = cg * g.sw[jd];
      if (!incoming) {
        v = comb_kernel(yx, yy, yz, g.px[jd], g.py[jd], g.pz[jd], g.nx[jd], g.ny[jd],
                        g.nz[jd], g.k, g.eta);
      } else {
        v = green(g.px[jd], g.py[jd], g.pz[jd], yx, yy, yz, g.k);
      }
      v = cscale(v, s);
    }
    reinterpret_cast<double2*>(M)[i + (int64_t)j * d.mmax] = v;
  }
}

void launch_assemble_id(const LevelDev& L, const Geometry& g, int b0, int nb, int mmax_max,
                        bool fp32, cudaStream_t st) {
  if (nb <= 0) return;
  dim3 grid((mmax_max + kIdRows - 1) / kIdRows, nb);
  if (fp32)
    FMMLU_LAUNCH("assemble_id", st, k_assemble_id<float2><<<grid, 256, 0, st>>>(L, g, b0));
  else
    FMMLU_LAUNCH("assemble_id", st, k_assemble_id<double2><<<grid, 256, 0, st>>>(L, g, b0));
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

__device__ __forceinline__ double2 elem(const LevelDev& L, const Geometry& g, const BoxDesc& d,
                                        Idx r, Idx c) {
  double2 v = entry(g, r.dof, c.dof);
  int cnt = 1 + d.ncnt;
  int64_t off = L.pairtab[d.pairtab + (int64_t)r.loc * cnt + c.loc];
  if (off >= 0) {
    int ld = r.loc == 0 ? d.a : L.cur_a0[L.nlist[d.nbeg + r.loc - 1]];
    v = cadd(v, L.delta[off + r.pos + (int64_t)c.pos * ld]);
  }
  return v;
}

constexpr int kElimTile = 4096;

__global__ void k_assemble_elim(LevelDev L, Geometry g, int b0) {
  int b = b0 + blockIdx.z;
  const BoxDesc d = L.desc[b];
  const BoxRun run = L.run[b];
  int a = d.a, s = run.s, n = run.n;
  if (s >= a) return;   // nothing to eliminate
  const int* perm = L.iarena + d.idx_off + d.a + d.nmax;
  const int* ndof = L.rows + d.rows_off + 3 * d.qmax;
  const int* npos = ndof + d.nmax;
  const int* nloc = npos + d.nmax;
  int64_t total = (int64_t)a * (a + n);
  int64_t e0 = (int64_t)blockIdx.x * kElimTile;
  if (e0 >= total) return;
  int64_t e1 = min(total, e0 + kElimTile);
  bool first = blockIdx.y == 0;
  double2* G1 = L.arena + d.G1_off;
  double2* G3 = L.arena + d.G3_off;
  int ld3 = a + d.nmax;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    if (first) {
      // G1: a x (a+n), rows B_piv, cols [S | N | R]
      int i = (int)(e % a), j = (int)(e / a);
      Idx r = bpiv(L, d, perm, i);
      Idx c = j < s ? bpiv(L, d, perm, j)
                    : (j < s + n ? Idx{ndof[j - s], nloc[j - s], npos[j - s]}
                                 : bpiv(L, d, perm, j - n));
      G1[i + (int64_t)j * a] = elem(L, g, d, r, c);
    } else {
      // G3: (a+n) x a, rows [S | N | R], cols B_piv
      int rows = a + n;
      int i = (int)(e % rows), j = (int)(e / rows);
      Idx r = i < s ? bpiv(L, d, perm, i)
                    : (i < s + n ? Idx{ndof[i - s], nloc[i - s], npos[i - s]}
                                 : bpiv(L, d, perm, i - n));
      Idx c = bpiv(L, d, perm, j);
      G3[i + (int64_t)j * ld3] = elem(L, g, d, r, c);
    }
  }
}

void launch_assemble_elim(const LevelDev& L, const Geometry& g, int b0, int nb, int amax,
                          int nmax_max, cudaStream_t st) {
  if (nb <= 0) return;
  int64_t total = (int64_t)amax * (amax + nmax_max);
  dim3 grid((unsigned)((total + kElimTile - 1) / kElimTile), 2, nb);
  FMMLU_LAUNCH("assemble_elim", st, k_assemble_elim<<<grid, 256, 0, st>>>(L, g, b0));
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
