// Row a2 in the paper's own KL variant (Sec. 3.1.1, Eq. KL-expansion and
// Eq. KL-expansion-deterministic; Sec. 4 parameters):
//   G(x, y) = G0 (1 + s Z(x, y)),   Z(x, y) = sum_k l_k(x) y_k,   y_k ~ U(-1, 1),
// the l_k the columns of a low-rank pivoted Cholesky factor of the Gaussian
// covariance C(x, x') = sigma2 exp(-|x - x'|^2 / ell^2).
//
// Set-up (once per context).  The factor is computed on the host over the cell
// centroids of a candidate grid (Harbrecht, Peters & Schneider 2012: greedy
// pivot = largest remainder diagonal, lowest index on ties; stop after M
// columns or when the remainder's trace falls below tol of the full trace);
// only the pivot points and the pivot rows of the factor are kept.  The
// columns then extend to any point by forward substitution (the Nystrom
// extension of a pivoted Cholesky factor),
//   l_m(x) = (C(x, x_{p_m}) - sum_{j<m} l_j(x) L_{p_m j}) / L_{p_m m},
// which one thread per cell evaluates on every level's centroids: the level's
// mode table Phi [cells][M] (FP64, and FP32 for the tensor cores), so that the
// fine and coarse fields of a pair are the same continuous field.
//
// Per sample the field is the contraction Z = Phi (s psi): the FP64 kernel
// below, or the tensor-core kernel of kl_tc.cu with Phi as its A operand.
#include <math.h>

#include <vector>

#include "internal.cuh"

namespace mlmc {

int pivoted_cholesky_host(int dim, const double* L, const int* n, double sigma2, double ell, int M,
                          double tol, std::vector<double>& xp, std::vector<double>& lpiv,
                          double* bound) {
  const int64_t cells = (int64_t)n[0] * (dim >= 2 ? n[1] : 1) * (dim >= 3 ? n[2] : 1);
  std::vector<double> X((size_t)cells * 3, 0.0);
  for (int64_t c = 0; c < cells; ++c) {
    const int64_t i = c % n[0], j = (c / n[0]) % (dim >= 2 ? n[1] : 1);
    const int64_t k = c / ((int64_t)n[0] * (dim >= 2 ? n[1] : 1));
    const int64_t ijk[3] = {i, j, k};
    for (int d = 0; d < dim; ++d) X[(size_t)c * 3 + d] = (ijk[d] + 0.5) * L[d] / n[d];
  }
  auto cov = [&](int64_t a, int64_t b) {
    double r2 = 0.0;
    for (int d = 0; d < dim; ++d) {
      const double t = X[(size_t)a * 3 + d] - X[(size_t)b * 3 + d];
      r2 += t * t;
    }
    return sigma2 * exp(-r2 / (ell * ell));
  };
  std::vector<double> rem((size_t)cells), fac((size_t)cells * M, 0.0);
  double tr0 = 0.0;
  for (int64_t c = 0; c < cells; ++c) { rem[c] = cov(c, c); tr0 += rem[c]; }
  std::vector<int64_t> piv;
  int m = 0;
  for (; m < M; ++m) {
    double tr = 0.0;
    for (int64_t c = 0; c < cells; ++c) tr += rem[c];
    if (tr <= tol * tr0) break;
    int64_t p = 0;
    for (int64_t c = 1; c < cells; ++c)
      if (rem[c] > rem[p]) p = c;
    if (!(rem[p] > 0.0)) break;
    const double sp = sqrt(rem[p]);
    piv.push_back(p);
    for (int64_t c = 0; c < cells; ++c) {
      double v = cov(c, p);
      for (int j = 0; j < m; ++j) v -= fac[(size_t)c * M + j] * fac[(size_t)p * M + j];
      fac[(size_t)c * M + m] = v / sp;
    }
    for (int64_t c = 0; c < cells; ++c) rem[c] -= fac[(size_t)c * M + m] * fac[(size_t)c * M + m];
    rem[p] = 0.0;
  }
  // max over the candidates of sum_k |L_ck|: the ellipticity bound's sup over
  // x, taken on the candidate grid so that every hierarchy sharing the grid
  // gets the same s_eff
  double b = 0.0;
  for (int64_t c = 0; c < cells; ++c) {
    double sa = 0.0;
    for (int j = 0; j < m; ++j) sa += fabs(fac[(size_t)c * M + j]);
    b = sa > b ? sa : b;
  }
  *bound = b;
  xp.assign((size_t)m * 3, 0.0);
  lpiv.assign((size_t)M * M, 0.0);
  for (int a = 0; a < m; ++a) {
    for (int d = 0; d < 3; ++d) xp[(size_t)a * 3 + d] = X[(size_t)piv[a] * 3 + d];
    for (int b = 0; b <= a; ++b) lpiv[(size_t)a * M + b] = fac[(size_t)piv[a] * M + b];
  }
  return m;
}

// One thread per cell: the forward substitution of the Nystrom extension,
// l kept in registers in chunks -- M is at most a few hundred, so the row of
// the cell lives in the output and is read back (L1) by the recursion.
__global__ void pc_eval_kernel(LevelDesc lv, int M, int m, double sigma2, double inv_ell2,
                               const double* __restrict__ xp, const double* __restrict__ lpiv,
                               double* __restrict__ phi64, float* __restrict__ phi32,
                               unsigned long long* bound) {
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double sum_abs = 0.0;
  if (cell < lv.cells) {
    const int i = (int)(cell % lv.n[0]);
    const int64_t r = cell / lv.n[0];
    const int j = (int)(r % lv.n[1]), k = (int)(r / lv.n[1]);
    const double x[3] = {(i + 0.5) * lv.h[0], (j + 0.5) * lv.h[1], (k + 0.5) * lv.h[2]};
    double* l = phi64 + cell * M;
    for (int a = 0; a < m; ++a) {
      double r2 = 0.0;
      for (int d = 0; d < lv.dim; ++d) {
        const double t = x[d] - xp[a * 3 + d];
        r2 += t * t;
      }
      double v = sigma2 * exp(-r2 * inv_ell2);
      for (int b = 0; b < a; ++b) v -= l[b] * lpiv[(int64_t)a * M + b];
      v /= lpiv[(int64_t)a * M + a];
      l[a] = v;
      sum_abs += fabs(v);
      if (phi32) phi32[cell * M + a] = (float)v;
    }
    for (int a = m; a < M; ++a) {
      l[a] = 0.0;
      if (phi32) phi32[cell * M + a] = 0.f;
    }
  }
  if (bound) {
    for (int o = 16; o > 0; o >>= 1) sum_abs = fmax(sum_abs, __shfl_xor_sync(0xffffffffu, sum_abs, o));
    if ((threadIdx.x & 31) == 0) atomicMax(bound, (unsigned long long)__double_as_longlong(sum_abs));
  }
}

cudaError_t launch_pc_eval(const LevelDesc& lv, int M, int m, double sigma2, double ell,
                           const double* xp, const double* lpiv, double* phi64, float* phi32,
                           unsigned long long* bound, cudaStream_t st) {
  if (lv.cells == 0) return cudaSuccess;
  const int bs = 128;
  pc_eval_kernel<<<(unsigned)((lv.cells + bs - 1) / bs), bs, 0, st>>>(
      lv, M, m, sigma2, 1.0 / (ell * ell), xp, lpiv, phi64, phi32, bound);
  return cudaGetLastError();
}

// One thread per (sample, cell); the coefficient row of the sample is reused
// by every cell through L1.
__global__ void kl_field_table_kernel(LevelDesc lv, int M, const double* __restrict__ coef,
                                      const double* __restrict__ phi64,
                                      const double* __restrict__ xi, int n, double* __restrict__ Z) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)n * lv.cells) return;
  const int s = (int)(g / lv.cells);
  const int64_t cell = g % lv.cells;
  const double* p = phi64 + cell * M;
  const double* y = xi + (int64_t)s * M;
  double z = 0.0;
  for (int k = 0; k < M; ++k) z += p[k] * (coef[k] * y[k]);
  Z[g] = z;
}

cudaError_t launch_kl_field_table(const LevelDesc& lv, int M, const double* coef,
                                  const double* phi64, const double* xi, int n, double* Z,
                                  cudaStream_t st) {
  const int64_t total = (int64_t)n * lv.cells;
  if (total == 0) return cudaSuccess;
  const int bs = 128;
  kl_field_table_kernel<<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>(lv, M, coef, phi64, xi, n, Z);
  return cudaGetLastError();
}

}  // namespace mlmc
