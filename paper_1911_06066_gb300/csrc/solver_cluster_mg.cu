// The multigrid-preconditioned instances of the cluster solver
// (solver_cluster.cuh with MG = true, global-memory layout; the V-cycle is in
// gmg.cuh), in a translation unit of their own so that the library's
// translation units compile in parallel.
#include "solver_cluster.cuh"

namespace mlmc {

cudaError_t launch_solve_cluster_gmg(const LevelDesc& lv, const Physics& ph, const SolverParams& sp,
                                     bool mixed, const ClusterPlan& pl, int n, const double* coef64,
                                     const float* coef32, double* slab, double* t_act,
                                     mlmc_sample_info* info, unsigned long long* counters,
                                     const ClusterGlobal& g, const MGDesc& mg, cudaStream_t st) {
  if (mixed) {
    if (lv.dim == 3)
      return launch_one<float, 3, true, true>(lv, ph, sp, pl, n, coef64, coef32, slab, t_act, info,
                                              counters, g, mg, st);
    return launch_one<float, 2, true, true>(lv, ph, sp, pl, n, coef64, coef32, slab, t_act, info,
                                            counters, g, mg, st);
  }
  if (lv.dim == 3)
    return launch_one<double, 3, true, true>(lv, ph, sp, pl, n, coef64, coef64, slab, t_act, info,
                                             counters, g, mg, st);
  return launch_one<double, 2, true, true>(lv, ph, sp, pl, n, coef64, coef64, slab, t_act, info,
                                           counters, g, mg, st);
}

}  // namespace mlmc
