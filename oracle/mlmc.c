/*
 * Oracle: Monte Carlo and multilevel Monte Carlo estimators (Sec. 3.1.2,
 * Eq. MC-estimator and Eq. MLMC-estimator, with u_{-1} = 0) on the activation
 * map, and the transfer of nodal fields between nested grids (Sec. 3.4; for
 * vertex-nested grids and a nodal quantity the transfer to the coarsest grid
 * is injection at the shared vertices).
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

void or_inject(const or_level* fine, const or_level* l0, const double* f, double* out) {
  int dim = fine->dim;
  int r = fine->n[0] / l0->n[0];
  int Nxf = fine->n[0] + 1, Nyf = dim >= 2 ? fine->n[1] + 1 : 1;
  int Nx0 = l0->n[0] + 1, Ny0 = dim >= 2 ? l0->n[1] + 1 : 1, Nz0 = dim == 3 ? l0->n[2] + 1 : 1;
  for (int k = 0; k < Nz0; ++k)
    for (int j = 0; j < Ny0; ++j)
      for (int i = 0; i < Nx0; ++i)
        out[(k * Ny0 + j) * Nx0 + i] = f[((size_t)(k * r) * Nyf + j * r) * Nxf + i * r];
}

/* Welford's running mean / sum of squared deviations, one update per sample. */
void or_welford_add(or_welford* w, int len, const double* y) {
  w->n += 1;
  for (int i = 0; i < len; ++i) {
    double d = y[i] - w->mean[i];
    w->mean[i] += d / (double)w->n;
    w->m2[i] += d * (y[i] - w->mean[i]);
  }
}

/*
 * One MLMC sample pair on level l (l = 0: a single coarsest-grid sample):
 * xi drawn once for (seed, l, id), the KL field evaluated on both grids, both
 * problems solved, activation maps injected to the coarsest grid, and
 *   y  = t_l - t_{l-1},       y2 = t_l^2 - t_{l-1}^2     (t_{-1} = 0).
 * kl = {sigma2, ell}.  Returns 0, or the failing solve's status.
 */
int or_sample_pair(const or_level* fine, const or_level* coarse, const or_level* l0,
                   double sigma2, double ell, int M, uint64_t seed, int level,
                   uint64_t sample_id, double* y, double* y2, int* newton_iters) {
  int n0 = or_nodes(l0);
  double* xi = malloc(sizeof(double) * M);
  or_xi(seed, level, sample_id, M, xi);
  const or_level* lv[2] = {fine, coarse};
  double* inj[2] = {malloc(sizeof(double) * n0), malloc(sizeof(double) * n0)};
  int ret = 0, iters = 0;
  for (int s = 0; s < 2; ++s) {
    if (!lv[s]) { for (int i = 0; i < n0; ++i) inj[s][i] = 0.0; continue; }
    int n = or_nodes(lv[s]);
    double* Z = malloc(sizeof(double) * or_cells(lv[s]));
    double* slab = malloc(sizeof(double) * (size_t)(lv[s]->m + 1) * n);
    double* t = malloc(sizeof(double) * n);
    or_kl_field(lv[s]->dim, lv[s]->L, lv[s]->n, sigma2, ell, M, 1, xi, Z);
    int rc = or_solve_sample(lv[s], Z, NULL, slab, t, NULL);
    if (rc < 0) ret = rc; else iters += rc;
    or_inject(lv[s], l0, t, inj[s]);
    free(Z); free(slab); free(t);
  }
  for (int i = 0; i < n0; ++i) {
    y[i] = inj[0][i] - inj[1][i];
    y2[i] = inj[0][i] * inj[0][i] - inj[1][i] * inj[1][i];
  }
  if (newton_iters) *newton_iters = iters;
  free(xi); free(inj[0]); free(inj[1]);
  return ret;
}
