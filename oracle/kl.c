/*
 * Oracle: truncated Karhunen-Loeve expansion of the log-conductivity
 * (Sec. 3.1.1, Eq. KL-expansion and KL-expansion-deterministic), in the variant
 * with the separable exponential covariance
 *     k(x, y) = sigma2 * prod_d exp(-|x_d - y_d| / ell)
 * whose eigenpairs are products of 1D eigenpairs with a closed form.
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * 1D eigenproblem of exp(-|x-y|/ell) on [-A, A] (the interval shifted to be
 * symmetric), c = 1/ell.  Eigenvalues lam = 2c/(w^2 + c^2) where w solves
 *   even (cosine) modes:  c - w tan(wA) = 0,   phi = cos(w x)/sqrt(A + sin(2wA)/(2w))
 *   odd  (sine)   modes:  w + c tan(wA) = 0,   phi = sin(w x)/sqrt(A - sin(2wA)/(2w))
 * Mode n (0-based, decreasing lam) has w A in (n pi/2, (n+1) pi/2) and is a
 * cosine mode for even n.  Roots are found by bisection on the pole-free forms
 * c cos(wA) - w sin(wA) and w cos(wA) + c sin(wA).
 *
 * Truncation: the M largest products; exact ties are broken by the sum of the
 * 1D indices, then lexicographically.  The field is evaluated at cell centroids.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

static double kl_char(int n, double w, double A, double c) {
  if (n % 2 == 0) return c * cos(w * A) - w * sin(w * A);
  return w * cos(w * A) + c * sin(w * A);
}

void or_kl_1d(double len, double ell, int n, double* omega, double* lam, double* nrm) {
  const double pi = 3.14159265358979323846;
  double A = 0.5 * len, c = 1.0 / ell;
  for (int k = 0; k < n; ++k) {
    double lo = (double)k * (pi / 2.0) / A, hi = (double)(k + 1) * (pi / 2.0) / A;
    double flo = kl_char(k, lo, A, c);
    for (int it = 0; it < 400; ++it) {
      double mid = 0.5 * (lo + hi);
      if (!(mid > lo && mid < hi)) break;
      double fm = kl_char(k, mid, A, c);
      if ((fm > 0.0) == (flo > 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
    }
    double w = 0.5 * (lo + hi);
    omega[k] = w;
    lam[k] = 2.0 * c / (w * w + c * c);
    double s = sin(2.0 * w * A) / (2.0 * w);
    nrm[k] = sqrt((k % 2 == 0) ? A + s : A - s);
  }
}

double or_kl_phi_1d(double len, int k, double omega, double nrm, double x) {
  double xs = x - 0.5 * len;
  return ((k % 2 == 0) ? cos(omega * xs) : sin(omega * xs)) / nrm;
}

typedef struct { double p; int i[3]; } cand;

static int cand_cmp(const void* pa, const void* pb) {
  const cand* a = (const cand*)pa; const cand* b = (const cand*)pb;
  if (a->p > b->p) return -1;
  if (a->p < b->p) return 1;
  int sa = a->i[0] + a->i[1] + a->i[2], sb = b->i[0] + b->i[1] + b->i[2];
  if (sa != sb) return sa < sb ? -1 : 1;
  for (int d = 0; d < 3; ++d) if (a->i[d] != b->i[d]) return a->i[d] < b->i[d] ? -1 : 1;
  return 0;
}

int or_kl_table(int dim, const double* L, double sigma2, double ell, int M,
                int* idx, double* sqrt_lam) {
  if (dim < 1 || dim > 3 || M < 1) return -1;
  double* lam[3]; double* om = malloc(sizeof(double) * M); double* nr = malloc(sizeof(double) * M);
  for (int d = 0; d < dim; ++d) { lam[d] = malloc(sizeof(double) * M); or_kl_1d(L[d], ell, M, om, lam[d], nr); }
  /* a tuple with (i+1)(j+1)(k+1) > M has at least M strictly larger products */
  long cap = 1; for (int d = 0; d < dim; ++d) cap *= M;
  long ncand = 0; cand* cs = NULL; long alloc = 0;
  int hi1 = M, hi2 = dim >= 2 ? M : 1, hi3 = dim >= 3 ? M : 1;
  for (int i = 0; i < hi1; ++i)
    for (int j = 0; j < hi2; ++j)
      for (int k = 0; k < hi3; ++k) {
        if ((long)(i + 1) * (j + 1) * (k + 1) > M) break;
        if (ncand == alloc) { alloc = alloc ? 2 * alloc : 1024; cs = realloc(cs, sizeof(cand) * alloc); }
        double p = lam[0][i];
        if (dim >= 2) p = p * lam[1][j];
        if (dim >= 3) p = p * lam[2][k];
        cs[ncand].p = p; cs[ncand].i[0] = i; cs[ncand].i[1] = j; cs[ncand].i[2] = k;
        ++ncand;
      }
  (void)cap;
  qsort(cs, ncand, sizeof(cand), cand_cmp);
  int ret = 0;
  if (ncand < M) ret = -2;
  for (int q = 0; q < M && q < ncand; ++q) {
    for (int d = 0; d < 3; ++d) idx[3 * q + d] = cs[q].i[d];
    sqrt_lam[q] = sqrt(sigma2 * cs[q].p);
  }
  free(cs); free(om); free(nr);
  for (int d = 0; d < dim; ++d) free(lam[d]);
  return ret;
}

int or_kl_field(int dim, const double* L, const int* n, double sigma2, double ell,
                int M, int nsamp, const double* xi, double* Z) {
  int* idx = malloc(sizeof(int) * 3 * M); double* sl = malloc(sizeof(double) * M);
  int rc = or_kl_table(dim, L, sigma2, ell, M, idx, sl);
  if (rc) { free(idx); free(sl); return rc; }
  /* 1D mode values at the cell centroids of each axis */
  double* phi[3] = {NULL, NULL, NULL};
  double* om = malloc(sizeof(double) * M); double* lm = malloc(sizeof(double) * M);
  double* nr = malloc(sizeof(double) * M);
  for (int d = 0; d < dim; ++d) {
    or_kl_1d(L[d], ell, M, om, lm, nr);
    phi[d] = malloc(sizeof(double) * (size_t)M * n[d]);
    double h = L[d] / n[d];
    for (int k = 0; k < M; ++k)
      for (int i = 0; i < n[d]; ++i)
        phi[d][(size_t)k * n[d] + i] = or_kl_phi_1d(L[d], k, om[k], nr[k], ((double)i + 0.5) * h);
  }
  int nx = n[0], ny = dim >= 2 ? n[1] : 1, nz = dim >= 3 ? n[2] : 1;
  size_t cells = (size_t)nx * ny * nz;
  for (int s = 0; s < nsamp; ++s) {
    const double* x = xi + (size_t)s * M;
    for (int kz = 0; kz < nz; ++kz)
      for (int jy = 0; jy < ny; ++jy)
        for (int ix = 0; ix < nx; ++ix) {
          double z = 0.0;
          for (int q = 0; q < M; ++q) {
            double v = phi[0][(size_t)idx[3 * q] * nx + ix];
            if (dim >= 2) v = v * phi[1][(size_t)idx[3 * q + 1] * ny + jy];
            if (dim >= 3) v = v * phi[2][(size_t)idx[3 * q + 2] * nz + kz];
            z += sl[q] * v * x[q];
          }
          Z[(size_t)s * cells + ((size_t)kz * ny + jy) * nx + ix] = z;
        }
  }
  for (int d = 0; d < dim; ++d) free(phi[d]);
  free(om); free(lm); free(nr); free(idx); free(sl);
  return 0;
}
