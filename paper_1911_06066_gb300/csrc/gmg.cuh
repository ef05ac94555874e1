// Row a7: geometric multigrid (GMG) preconditioner for the CG inner solves of
// the global-memory cluster layout (solver_cluster.cu).
//
// The paper preconditions its Krylov solver with ILU / block Jacobi on a CPU
// cluster (Sec. 3.5); here the inner system of every Newton step,
//   H d = -F,   H = K + diag(hm),   hm_i = M_i (1/dt - r'(u_i)),
// is preconditioned by one symmetric V-cycle on the SPD operator
//   A_0 = K + diag(|hm|),
// on a hierarchy of vertex-nested grids (coarse node I on fine node 2I along
// every halved axis, Sec. 3.4 -- the grids of the MLMC hierarchy are nested the
// same way):
//   * prolongation P: (tri)linear interpolation, weights 1 on coincident nodes
//     and 1/2 on the midpoints of a halved axis; restriction R = P^T;
//   * coarse stiffness K_{g+1} = R K_g P (Galerkin), evaluated exactly from the
//     fine couplings once per sample; coarse diagonal term d_{g+1} = R d_g (the
//     row sums of P^T diag(d_g) P, since the weights of P sum to one), once
//     per Newton iteration;
//   * smoother: l1-Jacobi, x <- x + W (b - A_g x) with W = diag(1 / (d_g +
//     sum_o |K_g[o]|)), nu sweeps before and after the coarse correction, from
//     x = 0 on the way down; the coarsest grid gets coarse_sweeps sweeps.
// The l1 diagonal bounds the spectrum of W A_g by 1, so every sweep is an
// A-norm contraction; with the same W before and after the correction the
// V-cycle is a symmetric positive definite operator, as CG requires.
//
// Layout: every level's vectors are contiguous per sample in global memory
// (workspace); CTA `rank` of the sample's cluster owns nodes
// [rank H_g, min((rank+1) H_g, N_g)), H_g = ceil(N_g / C), of every level; a
// cluster barrier (release / acquire at cluster scope) separates every sweep
// whose neighbours another CTA wrote.  Arithmetic is in the CG's precision KR
// (FP32 in the mixed path); the Galerkin products are accumulated in FP64.
#pragma once
#include <cooperative_groups.h>

#include "internal.cuh"

namespace mlmc {
namespace gmg {

namespace cgx = cooperative_groups;

__device__ __forceinline__ void barrier(cgx::cluster_group& cl, int C) {
  if (C == 1) __syncthreads(); else cl.sync();
}

struct Range {
  int lo, hi;
};
__device__ __forceinline__ Range range(int nodes, int C, int rank) {
  const int H = (nodes + C - 1) / C;
  const int lo = min(rank * H, nodes);
  return {lo, min(lo + H, nodes)};
}

__device__ __forceinline__ void coords(const MGLevel& L, int f, int& i, int& j, int& k) {
  i = f % L.N[0];
  const int r = f / L.N[0];
  j = r % L.N[1];
  k = r / L.N[1];
}

// sum_o K[o][f] x[f + offset(o)] over in-domain neighbours (couplings [o][nodes]).
template <int DIM, typename TA, typename TK, typename TX>
__device__ __forceinline__ TA apply_K(const TK* K, const MGLevel& L, int f, int i, int j, int k,
                                      const TX* x) {
  constexpr int NO = DIM == 3 ? 27 : (DIM == 2 ? 9 : 3);
  const int64_t n = L.nodes;
  const int N0 = L.N[0], N01 = L.N[0] * L.N[1];
  TA y = 0;
  const bool in = i > 0 && i < L.N[0] - 1 && j > 0 && j < L.N[1] - 1 &&
                  (DIM == 2 || (k > 0 && k < L.N[2] - 1));
  if (in) {
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const int dx = o % 3 - 1, dy = (DIM >= 2 ? (o / 3) % 3 - 1 : 0), dz = DIM == 3 ? o / 9 - 1 : 0;
      y += (TA)K[o * n + f] * (TA)x[f + dx + dy * N0 + dz * N01];
    }
  } else {
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const int dx = o % 3 - 1, dy = (DIM >= 2 ? (o / 3) % 3 - 1 : 0), dz = DIM == 3 ? o / 9 - 1 : 0;
      const int ii = i + dx, jj = j + dy, kk = k + dz;
      if (ii < 0 || ii >= L.N[0] || jj < 0 || jj >= L.N[1] || kk < 0 || kk >= L.N[2]) continue;
      y += (TA)K[o * n + f] * (TA)x[f + dx + dy * N0 + dz * N01];
    }
  }
  return y;
}

// Fine nodes of coarse coordinate c along one axis and their weights in
// column c of P: {2c-1, 2c, 2c+1} with {1/2, 1, 1/2} (clipped to the grid) on
// a halved axis, {c} with 1 otherwise.  Returns the count.
__device__ __forceinline__ int fine_support(int c, int halved, int Nf, int* idx, double* w) {
  if (!halved) { idx[0] = c; w[0] = 1.0; return 1; }
  int q = 0;
  if (2 * c - 1 >= 0) { idx[q] = 2 * c - 1; w[q] = 0.5; ++q; }
  idx[q] = 2 * c; w[q] = 1.0; ++q;
  if (2 * c + 1 < Nf) { idx[q] = 2 * c + 1; w[q] = 0.5; ++q; }
  return q;
}

// Coarse nodes interpolated at fine coordinate f along one axis and their
// weights in row f of P.  Returns the count.
__device__ __forceinline__ int coarse_support(int f, int halved, int* idx, double* w) {
  if (!halved) { idx[0] = f; w[0] = 1.0; return 1; }
  if ((f & 1) == 0) { idx[0] = f >> 1; w[0] = 1.0; return 1; }
  idx[0] = (f - 1) >> 1; w[0] = 0.5;
  idx[1] = (f + 1) >> 1; w[1] = 0.5;
  return 2;
}

// Galerkin couplings of coarse node c (coordinates ci, cj, ck) of level Lc
// from the couplings Kf of the next finer level Lf:
//   Kc[o'][c] = sum_{f, o} P[f][c] Kf[o][f] P[f + o][c + o'],
// and the l1 row sum sum_o' |Kc[o'][c]|.
template <int DIM, typename TK, typename KR>
__device__ void galerkin_node(const TK* Kf, const MGLevel& Lf, const MGLevel& Lc, int c, int ci,
                              int cj, int ck, KR* Kc, KR* ks) {
  constexpr int NO = DIM == 3 ? 27 : (DIM == 2 ? 9 : 3);
  double acc[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) acc[o] = 0.0;
  int fx[3], fy[3], fz[3];
  double wx[3], wy[3], wz[3];
  const int nx = fine_support(ci, Lf.cz[0], Lf.N[0], fx, wx);
  const int ny = fine_support(cj, Lf.cz[1], Lf.N[1], fy, wy);
  int nz = 1;
  fz[0] = 0; wz[0] = 1.0;
  if (DIM == 3) nz = fine_support(ck, Lf.cz[2], Lf.N[2], fz, wz);
  const int64_t nf = Lf.nodes;
  for (int a = 0; a < nz; ++a)
    for (int b = 0; b < ny; ++b)
      for (int e = 0; e < nx; ++e) {
        const double wf = wx[e] * wy[b] * wz[a];
        const int f = fx[e] + Lf.N[0] * (fy[b] + Lf.N[1] * fz[a]);
        for (int o = 0; o < NO; ++o) {
          const int dx = o % 3 - 1, dy = (DIM >= 2 ? (o / 3) % 3 - 1 : 0), dz = DIM == 3 ? o / 9 - 1 : 0;
          const int gi = fx[e] + dx, gj = fy[b] + dy, gk = fz[a] + dz;
          if (gi < 0 || gi >= Lf.N[0] || gj < 0 || gj >= Lf.N[1] || gk < 0 || gk >= Lf.N[2]) continue;
          const double kv = (double)Kf[o * nf + f];
          if (kv == 0.0) continue;
          int px[2], py[2], pz[2];
          double vx[2], vy[2], vz[2];
          const int mx = coarse_support(gi, Lf.cz[0], px, vx);
          const int my = coarse_support(gj, Lf.cz[1], py, vy);
          int mz = 1;
          pz[0] = 0; vz[0] = 1.0;
          if (DIM == 3) mz = coarse_support(gk, Lf.cz[2], pz, vz);
          const double s = wf * kv;
          for (int q = 0; q < mz; ++q)
            for (int r = 0; r < my; ++r)
              for (int t = 0; t < mx; ++t) {
                const int oo = (px[t] - ci + 1) + 3 * (py[r] - cj + 1) + (DIM == 3 ? 9 * (pz[q] - ck + 1) : 0);
                acc[oo] += s * vx[t] * vy[r] * vz[q];
              }
        }
      }
  double l1 = 0.0;
  const int64_t nc = Lc.nodes;
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    Kc[o * nc + c] = (KR)acc[o];
    l1 += fabs(acc[o]);
  }
  ks[c] = (KR)l1;
}

// (R v)[c] = sum_f P[f][c] v[f] (|v| with ABS) for coarse node c of Lc.
template <int DIM, bool ABS, typename TA, typename TV>
__device__ __forceinline__ TA restrict_node(const TV* v, const MGLevel& Lf, int ci, int cj, int ck) {
  int fx[3], fy[3], fz[3];
  double wx[3], wy[3], wz[3];
  const int nx = fine_support(ci, Lf.cz[0], Lf.N[0], fx, wx);
  const int ny = fine_support(cj, Lf.cz[1], Lf.N[1], fy, wy);
  int nz = 1;
  fz[0] = 0; wz[0] = 1.0;
  if (DIM == 3) nz = fine_support(ck, Lf.cz[2], Lf.N[2], fz, wz);
  TA s = 0;
  for (int a = 0; a < nz; ++a)
    for (int b = 0; b < ny; ++b)
      for (int e = 0; e < nx; ++e) {
        const TV x = v[fx[e] + Lf.N[0] * (fy[b] + Lf.N[1] * fz[a])];
        s += (TA)(wx[e] * wy[b] * wz[a]) * (TA)(ABS ? fabs(x) : x);
      }
  return s;
}

// (P x)[f] for fine node f (coordinates i, j, k) of Lf from coarse vector x of Lc.
template <int DIM, typename KR>
__device__ __forceinline__ KR prolong_node(const KR* x, const MGLevel& Lf, const MGLevel& Lc, int i,
                                           int j, int k) {
  int px[2], py[2], pz[2];
  double vx[2], vy[2], vz[2];
  const int mx = coarse_support(i, Lf.cz[0], px, vx);
  const int my = coarse_support(j, Lf.cz[1], py, vy);
  int mz = 1;
  pz[0] = 0; vz[0] = 1.0;
  if (DIM == 3) mz = coarse_support(k, Lf.cz[2], pz, vz);
  KR s = 0;
  for (int q = 0; q < mz; ++q)
    for (int r = 0; r < my; ++r)
      for (int t = 0; t < mx; ++t)
        s += (KR)(vx[t] * vy[r] * vz[q]) * x[px[t] + Lc.N[0] * (py[r] + Lc.N[1] * pz[q])];
  return s;
}

// Once per sample: level 0 l1 row sums from the FP64 fine couplings, then the
// Galerkin couplings and row sums of every coarser level.
template <int NT, int DIM, typename KR>
__device__ void build(const MGDesc& mg, KR* blk, const double* K0, cgx::cluster_group& cl, int C,
                      int rank) {
  constexpr int NO = DIM == 3 ? 27 : (DIM == 2 ? 9 : 3);
  {
    const MGLevel& L = mg.l[0];
    const Range r = range(L.nodes, C, rank);
    for (int f = r.lo + (int)threadIdx.x; f < r.hi; f += NT) {
      double s = 0.0;
      for (int o = 0; o < NO; ++o) s += fabs(K0[(int64_t)o * L.nodes + f]);
      blk[L.ks + f] = (KR)s;
    }
  }
  for (int g = 0; g + 1 < mg.G; ++g) {
    const MGLevel& Lf = mg.l[g];
    const MGLevel& Lc = mg.l[g + 1];
    const Range r = range(Lc.nodes, C, rank);
    for (int c = r.lo + (int)threadIdx.x; c < r.hi; c += NT) {
      int i, j, k;
      coords(Lc, c, i, j, k);
      if (g == 0) galerkin_node<DIM>(K0, Lf, Lc, c, i, j, k, blk + Lc.K, blk + Lc.ks);
      else galerkin_node<DIM>((const KR*)(blk + Lf.K), Lf, Lc, c, i, j, k, blk + Lc.K, blk + Lc.ks);
    }
    barrier(cl, C);
  }
}

// Once per Newton iteration, after hm (level 0's diagonal term, used as |hm|)
// is visible to the whole cluster: d_g = R d_{g-1} and the l1-Jacobi inverses
// of the coarse levels.  Ends with a barrier.
template <int NT, int DIM, typename KR>
__device__ void newton_setup(const MGDesc& mg, KR* blk, const KR* hm0, cgx::cluster_group& cl, int C,
                             int rank) {
  for (int g = 1; g < mg.G; ++g) {
    const MGLevel& Lf = mg.l[g - 1];
    const MGLevel& L = mg.l[g];
    const Range r = range(L.nodes, C, rank);
    for (int c = r.lo + (int)threadIdx.x; c < r.hi; c += NT) {
      int i, j, k;
      coords(L, c, i, j, k);
      const KR dv = g == 1 ? restrict_node<DIM, true, KR>(hm0, Lf, i, j, k)
                           : restrict_node<DIM, false, KR>(blk + Lf.d, Lf, i, j, k);
      blk[L.d + c] = dv;
      blk[L.inv + c] = (KR)1 / (dv + blk[L.ks + c]);
    }
    barrier(cl, C);
  }
}

// `sweeps` l1-Jacobi sweeps on level g for rhs B, from x = 0 (start == NULL)
// or from start (xa or xb of the level); returns the buffer holding the result.
// Every sweep ends with a barrier.
template <int NT, int DIM, typename KR>
__device__ KR* smooth(const MGLevel& L, const KR* K, const KR* dterm, bool abs_d, const KR* inv,
                      const KR* B, KR* xa, KR* xb, KR* start, int sweeps, cgx::cluster_group& cl,
                      int C, int rank) {
  const Range r = range(L.nodes, C, rank);
  KR* src = start;
  for (int s = 0; s < sweeps; ++s) {
    KR* dst = src == xa ? xb : xa;
    for (int f = r.lo + (int)threadIdx.x; f < r.hi; f += NT) {
      if (!src) {
        dst[f] = inv[f] * B[f];
      } else {
        int i, j, k;
        coords(L, f, i, j, k);
        const KR dv = abs_d ? (KR)fabs(dterm[f]) : dterm[f];
        const KR ax = apply_K<DIM, KR>(K, L, f, i, j, k, src) + dv * src[f];
        dst[f] = src[f] + inv[f] * (B[f] - ax);
      }
    }
    barrier(cl, C);
    src = dst;
  }
  return src;
}

// z = V(rhs): one V-cycle.  K0, hm0, inv0, rhs, z are the sample's level-0
// arrays (indexed by node); rhs must be visible to the whole cluster.  On
// return z holds this CTA's nodes only (the caller's next barrier publishes it).
template <int NT, int DIM, typename KR>
__device__ void vcycle(const MGDesc& mg, KR* blk, const KR* K0, const KR* hm0, const KR* inv0,
                       const KR* rhs, KR* z, cgx::cluster_group& cl, int C, int rank) {
  KR* X[MG_MAX_LEVELS];
  const int G = mg.G;
  for (int g = 0; g + 1 < G; ++g) {
    const MGLevel& L = mg.l[g];
    const KR* K = g ? blk + L.K : K0;
    const KR* dterm = g ? blk + L.d : hm0;
    const KR* inv = g ? blk + L.inv : inv0;
    const KR* B = g ? blk + L.b : rhs;
    X[g] = smooth<NT, DIM, KR>(L, K, dterm, g == 0, inv, B, blk + L.xa, blk + L.xb, nullptr, mg.nu,
                               cl, C, rank);
    const Range r = range(L.nodes, C, rank);
    KR* t = blk + L.t;
    for (int f = r.lo + (int)threadIdx.x; f < r.hi; f += NT) {
      int i, j, k;
      coords(L, f, i, j, k);
      const KR dv = g ? dterm[f] : (KR)fabs(dterm[f]);
      t[f] = B[f] - (apply_K<DIM, KR>(K, L, f, i, j, k, X[g]) + dv * X[g][f]);
    }
    barrier(cl, C);
    const MGLevel& Lc = mg.l[g + 1];
    const Range rc = range(Lc.nodes, C, rank);
    for (int c = rc.lo + (int)threadIdx.x; c < rc.hi; c += NT) {
      int i, j, k;
      coords(Lc, c, i, j, k);
      blk[Lc.b + c] = restrict_node<DIM, false, KR>(t, L, i, j, k);
    }
    // the coarse level's first sweep reads b only at the nodes this thread wrote
  }
  {
    const MGLevel& L = mg.l[G - 1];
    const KR* K = G > 1 ? blk + L.K : K0;
    const KR* dterm = G > 1 ? blk + L.d : hm0;
    const KR* inv = G > 1 ? blk + L.inv : inv0;
    const KR* B = G > 1 ? blk + L.b : rhs;
    X[G - 1] = smooth<NT, DIM, KR>(L, K, dterm, G == 1, inv, B, blk + L.xa, blk + L.xb, nullptr,
                                   mg.coarse_sweeps, cl, C, rank);
  }
  for (int g = G - 2; g >= 0; --g) {
    const MGLevel& L = mg.l[g];
    const MGLevel& Lc = mg.l[g + 1];
    const Range r = range(L.nodes, C, rank);
    KR* Xg = X[g];
    for (int f = r.lo + (int)threadIdx.x; f < r.hi; f += NT) {
      int i, j, k;
      coords(L, f, i, j, k);
      Xg[f] += prolong_node<DIM, KR>(X[g + 1], L, Lc, i, j, k);
    }
    barrier(cl, C);
    const KR* K = g ? blk + L.K : K0;
    const KR* dterm = g ? blk + L.d : hm0;
    const KR* inv = g ? blk + L.inv : inv0;
    const KR* B = g ? blk + L.b : rhs;
    X[g] = smooth<NT, DIM, KR>(L, K, dterm, g == 0, inv, B, blk + L.xa, blk + L.xb, Xg, mg.nu, cl,
                               C, rank);
  }
  const Range r0 = range(mg.l[0].nodes, C, rank);
  for (int f = r0.lo + (int)threadIdx.x; f < r0.hi; f += NT) z[f] = X[0][f];
}

}  // namespace gmg
}  // namespace mlmc
