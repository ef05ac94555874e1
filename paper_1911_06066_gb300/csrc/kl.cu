// Row a2: the truncated Karhunen-Loeve field Z (Sec. 3.1.1, Eq. KL-expansion and
// Eq. KL-expansion-deterministic) for the separable exponential covariance
//   k(x, y) = sigma2 prod_d exp(-|x_d - y_d| / ell).
// The multi-dimensional eigenpairs are products of 1D eigenpairs, which have a
// closed form (Ghanem & Spanos, Stochastic Finite Elements, Sec. 2.3): on
// [-A, A] with c = 1/ell and x = w A,
//   cosine modes:  x sin x - cA cos x = 0,  phi = cos(w t) / sqrt(A + sin(2wA)/(2w))
//   sine modes:    x cos x + cA sin x = 0,  phi = sin(w t) / sqrt(A - sin(2wA)/(2w))
//   lam = 2c / (w^2 + c^2);  1D mode n has x in (n pi/2, (n+1) pi/2), cosine for even n.
// The roots are found on the host by Newton's method safeguarded by the bracket.
// The M largest products are kept; exact ties (the (i,j)/(j,i) pairs of equal
// intervals) are ordered by the sum of the 1D indices, then lexicographically.
// Z is evaluated at cell centroids: Z = sum_q sqrt(lam_q) phi_q(centroid) xi_q.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace mlmc {

namespace {

double char_fn(int n, double x, double cA) {
  return (n % 2 == 0) ? x * sin(x) - cA * cos(x) : x * cos(x) + cA * sin(x);
}
double char_dfn(int n, double x, double cA) {
  return (n % 2 == 0) ? (1.0 + cA) * sin(x) + x * cos(x) : (1.0 + cA) * cos(x) - x * sin(x);
}

}  // namespace

// 1D eigenpairs of the unit-variance exponential kernel on an interval of
// length len: angular frequencies, eigenvalues and normalisation divisors.
void kl_1d_host(double len, double ell, int n, std::vector<double>& omega,
                std::vector<double>& lam, std::vector<double>& nrm) {
  const double pi = 3.141592653589793238462643;
  double A = 0.5 * len, c = 1.0 / ell, cA = c * A;
  omega.resize(n); lam.resize(n); nrm.resize(n);
  for (int k = 0; k < n; ++k) {
    double lo = k * (pi / 2.0), hi = (k + 1) * (pi / 2.0);
    double flo = char_fn(k, lo, cA);
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 300; ++it) {
      double f = char_fn(k, x, cA);
      if (f == 0.0) break;
      if ((f > 0.0) == (flo > 0.0)) lo = x; else hi = x;
      double step = f / char_dfn(k, x, cA);
      double xn = x - step;
      if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
      if (fabs(xn - x) <= 2e-16 * fabs(x) || hi - lo <= 4e-16 * hi) { x = xn; break; }
      x = xn;
    }
    double w = x / A;
    omega[k] = w;
    lam[k] = 2.0 * c / (w * w + c * c);
    double s = sin(2.0 * w * A) / (2.0 * w);
    nrm[k] = sqrt((k % 2 == 0) ? A + s : A - s);
  }
}

struct ModeSel { double p; int i[3]; };

// The M-term mode table.  Returns false if fewer than M candidates exist.
bool kl_table_host(int dim, const double* L, double sigma2, double ell, int M,
                   std::vector<int>& idx, std::vector<double>& sqrt_lam) {
  std::vector<double> lam[3], om, nr;
  for (int d = 0; d < dim; ++d) kl_1d_host(L[d], ell, M, om, lam[d], nr);
  std::vector<ModeSel> cand;
  // (i+1)(j+1)(k+1) > M implies at least M strictly larger products.
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < (dim >= 2 ? M : 1); ++j) {
      if ((long)(i + 1) * (j + 1) > M) break;
      for (int k = 0; k < (dim >= 3 ? M : 1); ++k) {
        if ((long)(i + 1) * (j + 1) * (k + 1) > M) break;
        double p = lam[0][i];
        if (dim >= 2) p *= lam[1][j];
        if (dim >= 3) p *= lam[2][k];
        cand.push_back({p, {i, j, k}});
      }
    }
  if ((int)cand.size() < M) return false;
  std::sort(cand.begin(), cand.end(), [](const ModeSel& a, const ModeSel& b) {
    if (a.p != b.p) return a.p > b.p;
    int sa = a.i[0] + a.i[1] + a.i[2], sb = b.i[0] + b.i[1] + b.i[2];
    if (sa != sb) return sa < sb;
    for (int d = 0; d < 3; ++d) if (a.i[d] != b.i[d]) return a.i[d] < b.i[d];
    return false;
  });
  idx.assign(3 * M, 0);
  sqrt_lam.assign(M, 0.0);
  for (int q = 0; q < M; ++q) {
    for (int d = 0; d < 3; ++d) idx[3 * q + d] = cand[q].i[d];
    sqrt_lam[q] = sqrt(sigma2 * cand[q].p);
  }
  return true;
}

// 1D mode values at the n_axis cell centroids of an axis: [n1d][n_axis].
void kl_phi_table_host(double len, double ell, int n1d, int n_axis, std::vector<double>& out) {
  std::vector<double> om, lam, nrm;
  kl_1d_host(len, ell, n1d, om, lam, nrm);
  out.assign((size_t)n1d * n_axis, 0.0);
  double h = len / n_axis, A = 0.5 * len;
  for (int k = 0; k < n1d; ++k)
    for (int i = 0; i < n_axis; ++i) {
      double t = (i + 0.5) * h - A;
      out[(size_t)k * n_axis + i] = ((k % 2 == 0) ? cos(om[k] * t) : sin(om[k] * t)) / nrm[k];
    }
}

// One thread per (sample, cell); the mode loop reads the tables through L1.
__global__ void kl_field_kernel(LevelDesc lv, int M, const double* __restrict__ sqrt_lam,
                                const int* __restrict__ idx, const double* __restrict__ phx,
                                const double* __restrict__ phy, const double* __restrict__ phz,
                                const double* __restrict__ xi, int n, double* __restrict__ Z) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)n * lv.cells) return;
  int s = (int)(g / lv.cells);
  int64_t cell = g % lv.cells;
  int i = (int)(cell % lv.n[0]);
  int64_t r = cell / lv.n[0];
  int j = (int)(r % lv.n[1]);
  int k = (int)(r / lv.n[1]);
  const double* x = xi + (int64_t)s * M;
  double z = 0.0;
  for (int q = 0; q < M; ++q) {
    double v = phx[(int64_t)idx[3 * q] * lv.n[0] + i];
    if (lv.dim >= 2) v *= phy[(int64_t)idx[3 * q + 1] * lv.n[1] + j];
    if (lv.dim >= 3) v *= phz[(int64_t)idx[3 * q + 2] * lv.n[2] + k];
    z += sqrt_lam[q] * v * x[q];
  }
  Z[g] = z;
}

cudaError_t launch_kl_field(const LevelDesc& lv, int M, const double* sqrt_lam, const int* idx,
                            const double* phi_x, const double* phi_y, const double* phi_z,
                            int n1d, const double* xi, int n, double* Z, cudaStream_t st) {
  (void)n1d;
  int64_t total = (int64_t)n * lv.cells;
  if (total == 0) return cudaSuccess;
  int bs = 256;
  kl_field_kernel<<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>(lv, M, sqrt_lam, idx, phi_x,
                                                                     phi_y, phi_z, xi, n, Z);
  return cudaGetLastError();
}

}  // namespace mlmc
