/*
 * Oracle: the paper's own KL variant (Sec. 3.1.1, Eq. KL-expansion and
 * Eq. KL-expansion-deterministic; Sec. 4 parameters):
 *   G(x, y) = G0 (1 + s Z(x, y)),   Z(x, y) = sum_k l_k(x) y_k,   y_k ~ U(-1, 1),
 * with l_k the columns of a low-rank pivoted Cholesky factor of the covariance
 * C(x, x') = sigma2 exp(-|x - x'|^2 / ell^2) (the Gaussian kernel), and s capped
 * so that s max_x sum_k |l_k(x)| <= delta (the uniform-ellipticity rule: then
 * G stays within G0 (1 +- delta) for every y in [-1, 1]^M).
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * Pivoted Cholesky (Harbrecht, Peters & Schneider, Appl. Numer. Math. 62, 2012):
 * on candidate points x_1..x_n, with the remainder diagonal d = diag(C), step m
 * takes the pivot p_m = argmax_i d_i (lowest index on ties), the column
 *   c_i = C(x_i, x_p) - sum_{j<m} L_ij L_pj,   L_im = c_i / sqrt(d_p),
 * and d_i -= L_im^2; it stops after M columns or when sum_i d_i <= tol sum_i C_ii.
 * The factor extends to any point x by the same recursion (the Nystrom
 * extension): l_m(x) = (C(x, x_{p_m}) - sum_{j<m} l_j(x) L_{p_m j}) / L_{p_m m},
 * which needs only the pivots and the pivot rows of L.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static double gauss_cov(int dim, const double* x, const double* y, double sigma2, double ell) {
  double r2 = 0.0;
  for (int d = 0; d < dim; ++d) r2 += (x[d] - y[d]) * (x[d] - y[d]);
  return sigma2 * exp(-r2 / (ell * ell));
}

int or_pivoted_cholesky(int dim, int n, const double* X, double sigma2, double ell, int M,
                        double tol, int* piv, double* Lpiv, double* L) {
  double* d = malloc(sizeof(double) * n);
  double* Lf = malloc(sizeof(double) * (size_t)n * M);
  double tr0 = 0.0;
  for (int i = 0; i < n; ++i) { d[i] = gauss_cov(dim, X + dim * i, X + dim * i, sigma2, ell); tr0 += d[i]; }
  int m = 0;
  for (; m < M; ++m) {
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += d[i];
    if (tr <= tol * tr0) break;
    int p = 0;
    for (int i = 1; i < n; ++i) if (d[i] > d[p]) p = i;
    if (!(d[p] > 0.0)) break;
    double sp = sqrt(d[p]);
    piv[m] = p;
    for (int i = 0; i < n; ++i) {
      double c = gauss_cov(dim, X + dim * i, X + dim * p, sigma2, ell);
      for (int j = 0; j < m; ++j) c -= Lf[(size_t)i * M + j] * Lf[(size_t)p * M + j];
      Lf[(size_t)i * M + m] = c / sp;
    }
    for (int i = 0; i < n; ++i) d[i] -= Lf[(size_t)i * M + m] * Lf[(size_t)i * M + m];
    d[p] = 0.0;
  }
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) Lpiv[a * M + b] = b <= a ? Lf[(size_t)piv[a] * M + b] : 0.0;
  if (L)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < M; ++j) L[(size_t)i * M + j] = j < m ? Lf[(size_t)i * M + j] : 0.0;
  free(d); free(Lf);
  return m;
}

void or_pc_eval(int dim, int ny, const double* Y, const double* Xp, double sigma2, double ell,
                int M, int m, const double* Lpiv, double* Phi) {
  for (int i = 0; i < ny; ++i) {
    double* l = Phi + (size_t)i * M;
    for (int k = 0; k < M; ++k) l[k] = 0.0;
    for (int k = 0; k < m; ++k) {
      double c = gauss_cov(dim, Y + dim * i, Xp + dim * k, sigma2, ell);
      for (int j = 0; j < k; ++j) c -= l[j] * Lpiv[k * M + j];
      l[k] = c / Lpiv[k * M + k];
    }
  }
}
