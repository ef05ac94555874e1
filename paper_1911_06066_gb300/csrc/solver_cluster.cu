// Host side of the cluster solver (solver_cluster.cuh): launch plans, kernel
// attributes and the launches of the Jacobi-preconditioned instances; the
// multigrid-preconditioned instances are compiled in solver_cluster_mg.cu.
#include <algorithm>

#include "solver_cluster.cuh"

namespace mlmc {

cudaError_t launch_solve_cluster_gmg(const LevelDesc& lv, const Physics& ph, const SolverParams& sp,
                                     bool mixed, const ClusterPlan& pl, int n, const double* coef64,
                                     const float* coef32, double* slab, double* t_act,
                                     mlmc_sample_info* info, unsigned long long* counters,
                                     const ClusterGlobal& g, const MGDesc& mg, cudaStream_t st);

// Shared-memory bytes of one CTA.
size_t cluster_smem_bytes(int dim, int nmax, bool mixed, bool coef_smem, int nt) {
  return smem_layout(dim, nmax, mixed ? 4 : 8, coef_smem, nt).total;
}


// Launch plan: the smallest cluster whose bands fit the shared memory (or the
// requested size want_C), and the block size.  Returns false when it does not
// fit.  With gm the vectors live in global memory: any C works, and C = 0
// picks clusters of 16 CTAs, or fewer for grids of at most 8192 nodes; nt is
// the block size of the gm layout (512, or 256: twice the samples per SM).
bool cluster_plan(const LevelDesc& lv, bool mixed, int want_C, ClusterPlan* plan, bool gm, int nt) {
  const int rowlen = lv.dim == 3 ? lv.N[0] * lv.N[1] : lv.N[0];
  const int nrows = lv.dim == 3 ? lv.N[2] : lv.N[1];   // 1 in one dimension: one row
  const size_t limit = 224 * 1024;
  if (gm) {
    int C = want_C;
    if (!C) {
      C = 16;
      while (C > 1 && (int64_t)C * 512 > lv.nodes) C /= 2;
    }
    plan->C = C;
    plan->H = (int)((lv.nodes + C - 1) / C);
    plan->nt = nt == 256 ? 256 : 512;
    plan->coef_smem = false;
    plan->gm = true;
    plan->smem = smem_layout(lv.dim, 0, mixed ? 4 : 8, false, plan->nt).total;
    return true;
  }
  for (int C = 1; C <= 16; C *= 2) {
    if (want_C && C != want_C) continue;
    int H = (nrows + C - 1) / C;
    int nmax = H * rowlen;
    if (nmax > 2400) continue;           // 512 threads x at most 5 nodes each
    int nt = 512;
    bool coef = cluster_smem_bytes(lv.dim, nmax, mixed, true, nt) <= limit;
    size_t bytes = cluster_smem_bytes(lv.dim, nmax, mixed, coef, nt);
    if (bytes > limit) continue;
    plan->C = C; plan->H = H; plan->nt = nt; plan->coef_smem = coef; plan->smem = bytes;
    plan->gm = false;
    return true;
  }
  return false;
}

template <typename KR, int DIM>
static cudaError_t launch_nt(const LevelDesc& lv, const Physics& ph, const SolverParams& sp,
                             const ClusterPlan& pl, int n, const double* coef64, const KR* coefK,
                             double* slab, double* t_act, mlmc_sample_info* info,
                             unsigned long long* counters, const ClusterGlobal& g,
                             const MGDesc& mg, cudaStream_t st) {
  if (pl.G > 0) {
    if (DIM != 3) return cudaErrorInvalidValue;   // the group layout serves the 3D grids
    return launch_one<KR, 3, true, false, true>(lv, ph, sp, pl, n, coef64, coefK, slab, t_act, info,
                                                counters, g, mg, st);
  }
  if (pl.gm && pl.nt == 256)
    return launch_one<KR, DIM, true, false, false, 256>(lv, ph, sp, pl, n, coef64, coefK, slab, t_act,
                                                        info, counters, g, mg, st);
  if (pl.gm)
    return launch_one<KR, DIM, true, false>(lv, ph, sp, pl, n, coef64, coefK, slab, t_act, info,
                                            counters, g, mg, st);
  return launch_one<KR, DIM, false, false>(lv, ph, sp, pl, n, coef64, coefK, slab, t_act, info,
                                           counters, g, mg, st);
}

template <typename KR, int DIM>
static cudaError_t preload_one(const ClusterPlan& pl) {
  if (pl.G > 0) return set_attrs<KR, 3, true, false, true>(pl);
  if (pl.gm && pl.nt == 256) return set_attrs<KR, DIM, true, false, false, 256>(pl);
  return pl.gm ? set_attrs<KR, DIM, true>(pl) : set_attrs<KR, DIM, false>(pl);
}

// Resident CTAs per SM of the group kernel and the SM count of the current
// device, cached per device and precision: the first query loads the kernel,
// so it runs before any graph capture (group_plan is called from the preloads).
template <typename KR>
static cudaError_t group_slots(size_t smem, int* per_sm, int* sms) {
  static int cache[64][2] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && cache[dev][0] > 0) {
    *per_sm = cache[dev][0];
    *sms = cache[dev][1];
    return cudaSuccess;
  }
  int nsm = 0, per = 0;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  auto kern = solve_cluster_kernel<KR, 3, 512, 5, true, false, true>;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 512, smem)) != cudaSuccess) return e;
  *per_sm = per;
  *sms = nsm;
  if (dev >= 0 && dev < 64) { cache[dev][0] = per; cache[dev][1] = nsm; }
  return cudaSuccess;
}

// G: the largest k * SMs / n (k = CTAs per SM, from the most the SMs hold
// down to 1) that keeps G <= S / 2 and at least `min_nodes` nodes per CTA --
// n G a whole multiple of the SM count, so that every SM runs the same number
// of CTAs and no group waits for a CTA that shares its SM with more others.
cudaError_t group_resident_samples(const LevelDesc& lv, bool mixed, int* m) {
  *m = 0;
  ClusterPlan pl;
  if (lv.dim != 3 || !cluster_plan(lv, mixed, 16, &pl, true)) return cudaSuccess;
  int per = 0, sms = 0;
  cudaError_t e = mixed ? group_slots<float>(pl.smem, &per, &sms) : group_slots<double>(pl.smem, &per, &sms);
  if (e != cudaSuccess) return e;
  *m = per * sms / 32;
  return cudaSuccess;
}

cudaError_t group_plan(const LevelDesc& lv, bool mixed, int n, bool force, ClusterPlan* plan, bool* ok) {
  *ok = false;
  if (lv.dim != 3 || n < 1 || n > GROUP_MAX_SAMPLES) return cudaSuccess;
  ClusterPlan pl;
  if (!cluster_plan(lv, mixed, 16, &pl, true)) return cudaSuccess;
  int per = 0, sms = 0;
  cudaError_t e = mixed ? group_slots<float>(pl.smem, &per, &sms) : group_slots<double>(pl.smem, &per, &sms);
  if (e != cudaSuccess) return e;
  const int S = per * sms;
  const int64_t min_nodes = force ? 512 : 1024;   // nodes per CTA at least
  int G = 0;
  for (int k = per; k >= 1 && G == 0; --k) {
    const int g = k * sms / n;
    if (g >= 1 && g <= S / 2 && g <= GROUP_MAX_CTAS && (int64_t)n * g <= GROUP_MAX_GRID &&
        lv.nodes / g >= min_nodes)
      G = g;
  }
  if (G == 0 && force) {   // small grids: as many CTAs as the nodes allow
    int64_t g = std::min<int64_t>(S / n, lv.nodes / min_nodes);
    g = std::min<int64_t>(g, std::min<int64_t>(S / 2, GROUP_MAX_CTAS));
    g = std::min<int64_t>(g, GROUP_MAX_GRID / n);
    G = (int)g;
  }
  if (G < (force ? 1 : 32)) return cudaSuccess;
  pl.C = G;
  pl.G = G;
  pl.H = (int)((lv.nodes + G - 1) / G);
  *plan = pl;
  *ok = true;
  return cudaSuccess;
}

template <typename KR, int DIM>
static cudaError_t max_clusters_one(const ClusterPlan& pl, int* count) {
  cudaError_t e = preload_one<KR, DIM>(pl);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = launch_cfg(pl, 1, nullptr, at);
  if (pl.G > 0) {   // the group layout needs every CTA resident: one group
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, solve_cluster_kernel<KR, 3, 512, 5, true, false, true>,
                                                      512, pl.smem);
    *count = per > 0 ? 1 : 0;
    return e;
  }
  if (pl.gm && pl.nt == 256)
    return cudaOccupancyMaxActiveClusters(count, solve_cluster_kernel<KR, DIM, 256, 5, true, false>, &cfg);
  return pl.gm ? cudaOccupancyMaxActiveClusters(count, solve_cluster_kernel<KR, DIM, 512, 5, true, false>, &cfg)
               : cudaOccupancyMaxActiveClusters(count, solve_cluster_kernel<KR, DIM, 512, 5, false, false>, &cfg);
}

cudaError_t preload_solve_cluster(const LevelDesc& lv, bool mixed, const ClusterPlan& pl) {
  if (mixed)
    return lv.dim == 3 ? preload_one<float, 3>(pl)
                       : (lv.dim == 2 ? preload_one<float, 2>(pl) : preload_one<float, 1>(pl));
  return lv.dim == 3 ? preload_one<double, 3>(pl)
                     : (lv.dim == 2 ? preload_one<double, 2>(pl) : preload_one<double, 1>(pl));
}

cudaError_t cluster_max_active(const LevelDesc& lv, bool mixed, const ClusterPlan& pl, int* count) {
  if (mixed)
    return lv.dim == 3   ? max_clusters_one<float, 3>(pl, count)
           : lv.dim == 2 ? max_clusters_one<float, 2>(pl, count)
                         : max_clusters_one<float, 1>(pl, count);
  return lv.dim == 3   ? max_clusters_one<double, 3>(pl, count)
         : lv.dim == 2 ? max_clusters_one<double, 2>(pl, count)
                       : max_clusters_one<double, 1>(pl, count);
}

cudaError_t launch_solve_cluster(const LevelDesc& lv, const Physics& ph, const SolverParams& sp,
                                 bool mixed, const ClusterPlan& pl, int n, const double* coef64,
                                 const float* coef32, double* slab, double* t_act,
                                 mlmc_sample_info* info, unsigned long long* counters,
                                 const ClusterGlobal& g, const MGDesc& mg, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (pl.gm && (!g.u || !g.F || !g.kr || !g.code)) return cudaErrorInvalidValue;
  if (pl.G > 0 && (!g.gsync || !g.gslot || mg.G > 0 || n > GROUP_MAX_SAMPLES ||
                   (int64_t)n * pl.G > GROUP_MAX_GRID))
    return cudaErrorInvalidValue;
  if (pl.gm && mg.G > 0) {
    if (!g.mg || mg.nu < 1 || mg.coarse_sweeps < 1 || mg.G > MG_MAX_LEVELS) return cudaErrorInvalidValue;
    return launch_solve_cluster_gmg(lv, ph, sp, mixed, pl, n, coef64, coef32, slab, t_act, info,
                                    counters, g, mg, st);
  }
  if (mixed) {
    if (lv.dim == 3)
      return launch_nt<float, 3>(lv, ph, sp, pl, n, coef64, coef32, slab, t_act, info, counters, g, mg, st);
    if (lv.dim == 2)
      return launch_nt<float, 2>(lv, ph, sp, pl, n, coef64, coef32, slab, t_act, info, counters, g, mg, st);
    return launch_nt<float, 1>(lv, ph, sp, pl, n, coef64, coef32, slab, t_act, info, counters, g, mg, st);
  }
  if (lv.dim == 3)
    return launch_nt<double, 3>(lv, ph, sp, pl, n, coef64, coef64, slab, t_act, info, counters, g, mg, st);
  if (lv.dim == 2)
    return launch_nt<double, 2>(lv, ph, sp, pl, n, coef64, coef64, slab, t_act, info, counters, g, mg, st);
  return launch_nt<double, 1>(lv, ph, sp, pl, n, coef64, coef64, slab, t_act, info, counters, g, mg, st);
}

// Multigrid hierarchy of grid lv (see MGDesc): level 0 is lv itself; every
// axis with an even cell count >= 2 is halved per level while the grid has
// more than 512 nodes.  Arrays are padded to 64 elements.
void mg_hierarchy(const LevelDesc& lv, int nu, int coarse_sweeps, MGDesc* mg) {
  *mg = MGDesc();
  mg->nu = nu;
  mg->coarse_sweeps = coarse_sweeps;
  const int NO = n_offsets(lv.dim);
  auto pad = [](int64_t x) { return (x + 63) & ~(int64_t)63; };
  int n[3] = {lv.n[0], lv.n[1], lv.n[2]};
  int64_t off = 0;
  int G = 0;
  while (G < MG_MAX_LEVELS) {
    MGLevel& L = mg->l[G];
    int64_t nodes = 1;
    for (int d = 0; d < 3; ++d) {
      L.n[d] = d < lv.dim ? n[d] : 1;
      L.N[d] = d < lv.dim ? n[d] + 1 : 1;
      nodes *= L.N[d];
    }
    L.nodes = (int)nodes;
    const int64_t np = pad(nodes);
    if (G == 0) {
      L.K = L.d = L.inv = L.b = -1;
      L.ks = off; off += np;
      L.xa = off; off += np;
      L.xb = off; off += np;
      L.t = off; off += np;
    } else {
      L.K = off; off += (int64_t)NO * np;
      L.ks = off; off += np;
      L.d = off; off += np;
      L.inv = off; off += np;
      L.xa = off; off += np;
      L.xb = off; off += np;
      L.b = off; off += np;
      L.t = off; off += np;
    }
    ++G;
    bool any = false;
    for (int d = 0; d < 3; ++d) {
      L.cz[d] = d < lv.dim && n[d] >= 2 && n[d] % 2 == 0;
      any = any || L.cz[d];
    }
    if (!any || nodes <= 512 || G == MG_MAX_LEVELS) {
      for (int d = 0; d < 3; ++d) L.cz[d] = 0;
      break;
    }
    for (int d = 0; d < 3; ++d)
      if (L.cz[d]) n[d] /= 2;
  }
  mg->G = G;
  mg->per_sample = pad(off);
}

}  // namespace mlmc
