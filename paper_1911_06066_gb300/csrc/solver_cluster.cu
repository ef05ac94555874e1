// Rows a4-a8 on thread-block clusters: the same per-sample Newton-CG sweep as
// solver.cu (Sec. 3.3, Eq. mono_disc; Sec. 3.5 -- the algorithm, its root
// selection rule and its stopping tests are documented there), laid out for
// GB300's distributed shared memory.
//
// Mapping.  One cluster of C CTAs owns one sample.  The node grid is cut into
// C bands of H whole rows (2D: rows of constant y; 3D: planes of constant z);
// CTA r owns rows [rH, min((r+1)H, rows)).  Every per-node vector of the sweep
// -- the FP64 state u (two slices), F, Ku, Kd and the CG vectors r, z, p, q, d,
// diag, diag^-1 (FP64, or FP32 in the mixed path), and optionally the FP32 /
// FP64 couplings used by the CG -- lives in the owning CTA's shared memory for
// the whole time sweep.  A stencil touching the row above or below the band
// reads the neighbour CTA's shared memory directly (DSMEM), so there is no
// halo copy; the barrier that publishes a vector is the one the algorithm
// needs anyway.  Dot products are reduced per warp, per CTA (fixed order),
// then across the cluster by reading every CTA's partial in rank order, so the
// result is identical on all CTAs and deterministic.  Per CG iteration the
// cluster synchronises three times (p^T H p, r^T z, and the new p).
//
// Only the per-sample couplings (read once per Newton step by the residual)
// and the outputs stay in global memory.
#include <cooperative_groups.h>
#include <math.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace mlmc {

namespace {

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Band geometry of this CTA.
struct Band {
  int C, rank, H, row0, row1, rowlen, nrows, nb, nmax;
  int N0, N1, N2;
};

// A per-node shared-memory vector and the same vector of the two neighbour
// CTAs (nullptr at the ends of the cluster).
template <typename T>
struct View {
  T* loc;
  const T* prev;
  const T* next;
};

template <typename T>
__device__ __forceinline__ View<T> make_view(cg::cluster_group& cl, const Band& b, T* p) {
  View<T> v;
  v.loc = p;
  v.prev = b.rank > 0 ? cl.map_shared_rank(p, b.rank - 1) : nullptr;
  v.next = b.rank < b.C - 1 ? cl.map_shared_rank(p, b.rank + 1) : nullptr;
  return v;
}

// sum_o c[o] v[neighbour o] for the node (i, j, k); out-of-domain neighbours
// have zero couplings and are skipped.  c(o) returns the coupling.
template <int DIM, typename TA, typename TV, typename CF>
__device__ __forceinline__ TA stencil_band(const Band& b, const View<TV>& v, int i, int j, int k,
                                           CF c) {
  TA y = 0;
#pragma unroll
  for (int o = 0; o < (DIM == 3 ? 27 : 9); ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = DIM == 3 ? o / 9 - 1 : 0;
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    if (ii < 0 || ii >= b.N0 || jj < 0 || jj >= b.N1 || kk < 0 || kk >= b.N2) continue;
    const int row = DIM == 3 ? kk : jj;
    const int inrow = DIM == 3 ? jj * b.N0 + ii : ii;
    TV val;
    if (row >= b.row0 && row < b.row1) val = v.loc[(row - b.row0) * b.rowlen + inrow];
    else if (row < b.row0) val = v.prev[(b.H - 1) * b.rowlen + inrow];
    else val = v.next[inrow];
    y += (TA)c(o) * (TA)val;
  }
  return y;
}

// Deterministic sum / max over the cluster; every thread of every CTA gets it.
template <int NT>
__device__ double cluster_reduce(double v, bool is_max, double* red, double* slot, int& par,
                                 cg::cluster_group& cl, int C) {
  v = is_max ? wmax(v) : wsum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = red[0];
    for (int w = 1; w < NT / 32; ++w) t = is_max ? fmax(t, red[w]) : t + red[w];
    slot[par] = t;
  }
  double tot;
  if (C == 1) {
    __syncthreads();
    tot = slot[par];
  } else {
    cl.sync();
    tot = *cl.map_shared_rank(&slot[par], 0);
    for (int q = 1; q < C; ++q) {
      double x = *cl.map_shared_rank(&slot[par], q);
      tot = is_max ? fmax(tot, x) : tot + x;
    }
  }
  par ^= 1;
  return tot;
}

__device__ __forceinline__ void cluster_barrier(cg::cluster_group& cl, int C) {
  if (C == 1) __syncthreads(); else cl.sync();
}

}  // namespace

// Byte offsets of the per-CTA shared-memory arrays; every array starts on a
// 16-byte boundary.  Used by the kernel's carve-up and the host's sizing.
struct SmemLayout {
  size_t u0, u1, F, Ku, Kd, r, z, p, q, d, hm, pinv, cs, red, slot, total;
};

__host__ __device__ inline SmemLayout smem_layout(int dim, int nmax, int kr, bool coef_smem, int nt) {
  SmemLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = (o + bytes + 15) & ~(size_t)15;
    return at;
  };
  const size_t n8 = (size_t)nmax * 8, nk = (size_t)nmax * kr;
  L.u0 = take(n8); L.u1 = take(n8); L.F = take(n8); L.Ku = take(n8); L.Kd = take(n8);
  L.r = take(nk); L.z = take(nk); L.p = take(nk); L.q = take(nk); L.d = take(nk);
  L.hm = take(nk); L.pinv = take(nk);
  L.cs = take(coef_smem ? (size_t)n_offsets(dim) * nk : 0);
  L.red = take((size_t)(nt / 32) * 8);
  L.slot = take(2 * 8);
  L.total = o;
  return L;
}

// Shared-memory bytes of one CTA.
size_t cluster_smem_bytes(int dim, int nmax, bool mixed, bool coef_smem, int nt) {
  return smem_layout(dim, nmax, mixed ? 4 : 8, coef_smem, nt).total;
}

template <typename KR, int DIM, int NT>
__global__ void __launch_bounds__(NT, 1)
solve_cluster_kernel(LevelDesc lv, Physics ph, SolverParams sp, const double* __restrict__ coef64,
                     const KR* __restrict__ coefK, int H, int coef_smem, double* slab,
                     double* t_act, mlmc_sample_info* info, unsigned long long* counters) {
  constexpr int NO = DIM == 3 ? 27 : 9;
  cg::cluster_group cl = cg::this_cluster();
  Band b;
  b.C = (int)cl.num_blocks();
  b.rank = (int)cl.block_rank();
  b.N0 = lv.N[0]; b.N1 = lv.N[1]; b.N2 = lv.N[2];
  b.rowlen = DIM == 3 ? b.N0 * b.N1 : b.N0;
  b.nrows = DIM == 3 ? b.N2 : b.N1;
  b.H = H;
  b.row0 = min(b.rank * H, b.nrows);
  b.row1 = min(b.row0 + H, b.nrows);
  b.nb = (b.row1 - b.row0) * b.rowlen;
  b.nmax = H * b.rowlen;
  const int s = blockIdx.x / b.C;
  const int N = (int)lv.nodes;
  const int base = b.row0 * b.rowlen;
  const int nmax = b.nmax;

  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(DIM, nmax, (int)sizeof(KR), coef_smem != 0, NT);
  double* ubuf0 = (double*)(smem + L.u0);
  double* ubuf1 = (double*)(smem + L.u1);
  double* F = (double*)(smem + L.F);
  double* Ku = (double*)(smem + L.Ku);
  double* Kd = (double*)(smem + L.Kd);
  KR* r = (KR*)(smem + L.r);
  KR* z = (KR*)(smem + L.z);
  KR* p = (KR*)(smem + L.p);
  KR* q = (KR*)(smem + L.q);
  KR* d = (KR*)(smem + L.d);
  KR* hm = (KR*)(smem + L.hm);
  KR* pinv = (KR*)(smem + L.pinv);
  KR* cs = (KR*)(smem + L.cs);                             // couplings [NO][nmax] if coef_smem
  double* red = (double*)(smem + L.red);
  double* slot = (double*)(smem + L.slot);
  int par = 0;

  const double* c64 = coef64 + (int64_t)s * NO * N;
  const KR* cKg = coefK + (int64_t)s * NO * N;
  double* ta = t_act + (int64_t)s * N;
  double* sl = slab ? slab + (int64_t)s * (lv.m + 1) * N : nullptr;
  const double dt = lv.dt, inv_dt = 1.0 / lv.dt;

  cl.sync();   // every CTA of the cluster is resident before any DSMEM access

  // couplings of the CG into shared memory; initial state
  if (coef_smem)
    for (int o = 0; o < NO; ++o)
      for (int a = threadIdx.x; a < b.nb; a += NT) cs[o * nmax + a] = cKg[(int64_t)o * N + base + a];
  for (int a = threadIdx.x; a < b.nb; a += NT) {
    int A = base + a, i, j, k;
    node_ijk(lv, A, i, j, k);
    double x[3] = {i * lv.h[0], j * lv.h[1], k * lv.h[2]};
    double r2 = 0.0;
    for (int dd = 0; dd < DIM; ++dd) r2 += (x[dd] - ph.stim_c[dd]) * (x[dd] - ph.stim_c[dd]);
    double v = r2 < ph.stim_r2 ? 1.0 : 0.0;
    ubuf0[a] = v;
    ta[A] = v >= 0.5 ? 0.0 : -1.0;
    if (sl) sl[A] = v;
  }
  const View<KR> pv = make_view(cl, b, p);
  const View<KR> dv = make_view(cl, b, d);
  const View<double> uv0 = make_view(cl, b, ubuf0);
  const View<double> uv1 = make_view(cl, b, ubuf1);
  auto c64f = [&](int A) { return [=](int o) { return c64[(int64_t)o * N + A]; }; };

  int status = MLMC_OK, failed_step = 0;
  int newton_total = 0, cg_total = 0, trunc_total = 0, halvings = 0, max_newton = 0;
  for (int step = 1; step <= lv.m; ++step) {
    double* u = (step & 1) ? ubuf1 : ubuf0;
    const double* up = (step & 1) ? ubuf0 : ubuf1;
    const View<double>& uv = (step & 1) ? uv1 : uv0;
    for (int a = threadIdx.x; a < b.nb; a += NT) u[a] = up[a];
    cluster_barrier(cl, b.C);
    bool conv = false, lin_fail = false;
    int it;
    for (it = 1; it <= sp.newton_max; ++it) {
      double rz_loc = 0.0;
      for (int a = threadIdx.x; a < b.nb; a += NT) {
        int A = base + a, i, j, k;
        node_ijk(lv, A, i, j, k);
        double mA = lumped_mass(lv, i, j, k);
        double uA = u[a];
        double ku = stencil_band<DIM, double>(b, uv, i, j, k, c64f(A));
        Ku[a] = ku;
        double f = ku + mA * inv_dt * (uA - up[a]) - mA * rxn(ph, uA);
        F[a] = f;
        double hmA = mA / dt - mA * rxn_d(ph, uA);
        double pvv = 1.0 / fabs(hmA + c64[(int64_t)centre_offset(DIM) * N + A]);
        KR rv = (KR)(-f);
        KR zv = (KR)pvv * rv;
        hm[a] = (KR)hmA;
        pinv[a] = (KR)pvv;
        r[a] = rv; z[a] = zv; p[a] = zv; d[a] = (KR)0;
        rz_loc += (double)(rv * zv);
      }
      double rz = cluster_reduce<NT>(rz_loc, false, red, slot, par, cl, b.C);
      const double r0 = sqrt(rz);
      int cgi = 0;
      bool truncated = false;
      if (r0 > 0.0) {
        bool ok = false;
        for (cgi = 1; cgi <= sp.lin_max; ++cgi) {
          KR pq_loc = 0;
          for (int a = threadIdx.x; a < b.nb; a += NT) {
            int A = base + a, i, j, k;
            node_ijk(lv, A, i, j, k);
            KR hp;
            if (coef_smem)
              hp = stencil_band<DIM, KR>(b, pv, i, j, k, [=](int o) { return cs[o * nmax + a]; });
            else
              hp = stencil_band<DIM, KR>(b, pv, i, j, k, [=](int o) { return cKg[(int64_t)o * N + A]; });
            KR qv = hp + hm[a] * p[a];
            q[a] = qv;
            pq_loc += p[a] * qv;
          }
          double pq = cluster_reduce<NT>((double)pq_loc, false, red, slot, par, cl, b.C);
          if (pq <= 0.0) {
            truncated = true;
            if (cgi == 1)
              for (int a = threadIdx.x; a < b.nb; a += NT) d[a] = z[a];
            ok = true;
            break;
          }
          const KR alpha = (KR)(rz / pq);
          KR rzn_loc = 0;
          for (int a = threadIdx.x; a < b.nb; a += NT) {
            d[a] += alpha * p[a];
            KR rv = r[a] - alpha * q[a];
            KR zv = pinv[a] * rv;
            r[a] = rv;
            z[a] = zv;
            rzn_loc += rv * zv;
          }
          double rz_new = cluster_reduce<NT>((double)rzn_loc, false, red, slot, par, cl, b.C);
          if (sqrt(rz_new) <= sp.lin_rtol * r0) { ok = true; break; }
          const KR beta = (KR)(rz_new / rz);
          for (int a = threadIdx.x; a < b.nb; a += NT) p[a] = z[a] + beta * p[a];
          cluster_barrier(cl, b.C);
          rz = rz_new;
        }
        if (!ok) { lin_fail = true; cgi = sp.lin_max; }
      }
      cg_total += cgi;
      trunc_total += truncated ? 1 : 0;
      if (lin_fail) break;
      double dm_loc = 0.0;
      for (int a = threadIdx.x; a < b.nb; a += NT) dm_loc = fmax(dm_loc, fabs((double)d[a]));
      const double dmax = cluster_reduce<NT>(dm_loc, true, red, slot, par, cl, b.C);
      double alpha = 1.0;
      if (dmax > sp.step_max) alpha = sp.step_max / dmax;
      if (dmax > sp.newton_tol && dmax > sp.ls_full_step) {
        double gd_loc = 0.0;
        for (int a = threadIdx.x; a < b.nb; a += NT) {
          int A = base + a, i, j, k;
          node_ijk(lv, A, i, j, k);
          Kd[a] = stencil_band<DIM, double>(b, dv, i, j, k, c64f(A));
          gd_loc += F[a] * (double)d[a];
        }
        const double gd = cluster_reduce<NT>(gd_loc, false, red, slot, par, cl, b.C);
        for (int h = 0; h < 40; ++h) {
          double e_loc = 0.0;
          for (int a = threadIdx.x; a < b.nb; a += NT) {
            int A = base + a, i, j, k;
            node_ijk(lv, A, i, j, k);
            double mA = lumped_mass(lv, i, j, k);
            double uA = u[a], w = alpha * (double)d[a], v = uA + w;
            double sm = v + uA, q2 = v * v + uA * uA, q3 = v * v + v * uA + uA * uA;
            double rdiff = ph.c * w * (-sm * q2 / 4.0 + (1.0 + ph.a) * q3 / 3.0 - ph.a * sm / 2.0);
            e_loc += mA * w * (2.0 * (uA - up[a]) + w) / (2.0 * dt) + w * Ku[a] +
                     0.5 * w * alpha * Kd[a] - mA * rdiff;
          }
          double dE = cluster_reduce<NT>(e_loc, false, red, slot, par, cl, b.C);
          if (dE <= 1e-4 * alpha * gd) break;
          alpha *= 0.5;
          ++halvings;
        }
      }
      for (int a = threadIdx.x; a < b.nb; a += NT) u[a] += alpha * (double)d[a];
      cluster_barrier(cl, b.C);
      if (dmax <= sp.newton_tol) { conv = true; break; }
    }
    int used = it > sp.newton_max ? sp.newton_max : it;
    newton_total += used;
    max_newton = used > max_newton ? used : max_newton;
    if (!conv) { status = MLMC_ERR_NOT_CONVERGED; failed_step = step; break; }
    for (int a = threadIdx.x; a < b.nb; a += NT) {
      int A = base + a;
      if (ta[A] < 0.0 && u[a] >= 0.5) {
        double uo = up[a];
        ta[A] = (double)(step - 1) * dt + dt * (0.5 - uo) / (u[a] - uo);
      }
      if (sl) sl[(int64_t)step * N + A] = u[a];
    }
  }
  for (int a = threadIdx.x; a < b.nb; a += NT)
    if (ta[base + a] < 0.0) ta[base + a] = lv.T;
  if (b.rank == 0 && threadIdx.x == 0) {
    if (counters) {
      if (status != MLMC_OK) atomicAdd(counters, 1ull);
      atomicAdd(counters + 1, (unsigned long long)cg_total * (unsigned long long)N);
      atomicAdd(counters + 2, (unsigned long long)newton_total * (unsigned long long)N);
      atomicAdd(counters + 3, (unsigned long long)trunc_total);
      atomicAdd(counters + 4, (unsigned long long)halvings);
    }
    if (info) {
      mlmc_sample_info o;
      o.status = status; o.failed_step = failed_step; o.newton_iters = newton_total;
      o.cg_iters = cg_total; o.truncations = trunc_total; o.halvings = halvings;
      o.max_newton = max_newton; o.pad = 0;
      info[s] = o;
    }
  }
  cl.sync();   // no CTA leaves while a neighbour may still read its shared memory
}

// Launch plan: the smallest cluster whose bands fit the shared memory, and the
// block size.  Returns false when no cluster size up to 16 fits.
bool cluster_plan(const LevelDesc& lv, bool mixed, ClusterPlan* plan) {
  const int rowlen = lv.dim == 3 ? lv.N[0] * lv.N[1] : lv.N[0];
  const int nrows = lv.dim == 3 ? lv.N[2] : lv.N[1];
  const size_t limit = 200 * 1024;
  for (int C = 1; C <= 16; C *= 2) {
    int H = (nrows + C - 1) / C;
    int nmax = H * rowlen;
    if (nmax > 2400 && C < 16) continue;
    int nt = nmax <= 1200 ? 512 : 1024;
    bool coef = cluster_smem_bytes(lv.dim, nmax, mixed, true, nt) <= limit;
    size_t bytes = cluster_smem_bytes(lv.dim, nmax, mixed, coef, nt);
    if (bytes > limit) continue;
    plan->C = C; plan->H = H; plan->nt = nt; plan->coef_smem = coef; plan->smem = bytes;
    return true;
  }
  return false;
}

template <typename KR, int DIM, int NT>
static cudaError_t launch_one(const LevelDesc& lv, const Physics& ph, const SolverParams& sp,
                              const ClusterPlan& pl, int n, const double* coef64, const KR* coefK,
                              double* slab, double* t_act, mlmc_sample_info* info,
                              unsigned long long* counters, cudaStream_t st) {
  auto kern = solve_cluster_kernel<KR, DIM, NT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return e;
  if (pl.C > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * pl.C));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = pl.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, lv, ph, sp, coef64, coefK, pl.H, pl.coef_smem ? 1 : 0, slab,
                            t_act, info, counters);
}

template <typename KR, int DIM>
static cudaError_t launch_nt(const LevelDesc& lv, const Physics& ph, const SolverParams& sp,
                             const ClusterPlan& pl, int n, const double* coef64, const KR* coefK,
                             double* slab, double* t_act, mlmc_sample_info* info,
                             unsigned long long* counters, cudaStream_t st) {
  if (pl.nt == 1024)
    return launch_one<KR, DIM, 1024>(lv, ph, sp, pl, n, coef64, coefK, slab, t_act, info, counters, st);
  return launch_one<KR, DIM, 512>(lv, ph, sp, pl, n, coef64, coefK, slab, t_act, info, counters, st);
}

cudaError_t launch_solve_cluster(const LevelDesc& lv, const Physics& ph, const SolverParams& sp,
                                 bool mixed, const ClusterPlan& pl, int n, const double* coef64,
                                 const float* coef32, double* slab, double* t_act,
                                 mlmc_sample_info* info, unsigned long long* counters,
                                 cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (mixed) {
    if (lv.dim == 3)
      return launch_nt<float, 3>(lv, ph, sp, pl, n, coef64, coef32, slab, t_act, info, counters, st);
    return launch_nt<float, 2>(lv, ph, sp, pl, n, coef64, coef32, slab, t_act, info, counters, st);
  }
  if (lv.dim == 3)
    return launch_nt<double, 3>(lv, ph, sp, pl, n, coef64, coef64, slab, t_act, info, counters, st);
  return launch_nt<double, 2>(lv, ph, sp, pl, n, coef64, coef64, slab, t_act, info, counters, st);
}

}  // namespace mlmc
