// Rows a9-a10: level-pair differences of the activation map on the coarsest
// grid and the MC / MLMC estimators (Sec. 3.1.2, Eq. MC-estimator and
// Eq. MLMC-estimator, u_{-1} = 0).
//
// Transfer (Sec. 3.4): the grids are vertex-nested, so a nodal field of level
// l is restricted to level 0 by injection at the shared vertices
// (node (i,j,k) of level 0 is node (i r, j r, k r) of level l, r = 2^l).
//
// Accumulation: per level and coarsest-grid node, a running (n, mean, M2) of
// Y_l = t_l - t_{l-1} and a running mean of Y2_l = t_l^2 - t_{l-1}^2.  A batch
// is reduced in sample order (two passes: mean, then squared deviations) and
// merged with the pairwise update of Chan, Golub & LeVeque (1979):
//   delta = mean_b - mean_a,  n = n_a + n_b,
//   mean = mean_a + delta n_b / n,  M2 = M2_a + M2_b + delta^2 n_a n_b / n.
#include <math.h>

#include "internal.cuh"

namespace mlmc {

__global__ void iota_kernel(uint64_t first, int n, uint64_t* ids) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ids[i] = first + (uint64_t)i;
}

cudaError_t launch_iota(uint64_t first, int n, uint64_t* ids, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  iota_kernel<<<(n + 255) / 256, 256, 0, st>>>(first, n, ids);
  return cudaGetLastError();
}

__device__ inline int64_t injected_node(const LevelDesc& l0, const LevelDesc& lf, int64_t A0) {
  int r = lf.n[0] / l0.n[0];
  int i, j, k;
  node_ijk(l0, A0, i, j, k);
  return ((int64_t)(k * r) * lf.N[1] + (int64_t)j * r) * lf.N[0] + (int64_t)i * r;
}

// cens (device, may be NULL): count of injected fine activation times equal to
// T (never activated by the end time), warp-aggregated.
__global__ void pair_diff_kernel(LevelDesc l0, LevelDesc lf, LevelDesc lc, bool has_coarse,
                                 const double* __restrict__ tf, const double* __restrict__ tc,
                                 int n, double* __restrict__ y, double* __restrict__ y2,
                                 unsigned long long* cens) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = g < (int64_t)n * l0.nodes;
  bool censored = false;
  if (valid) {
    const int s = (int)(g / l0.nodes);
    const int64_t A0 = g % l0.nodes;
    const double a = tf[(int64_t)s * lf.nodes + injected_node(l0, lf, A0)];
    const double b = has_coarse ? tc[(int64_t)s * lc.nodes + injected_node(l0, lc, A0)] : 0.0;
    y[g] = a - b;
    y2[g] = a * a - b * b;
    censored = a >= lf.T;
  }
  if (cens) {
    const unsigned m = __ballot_sync(0xffffffffu, censored);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(cens, (unsigned long long)__popc(m));
  }
}

cudaError_t launch_pair_diff(const LevelDesc& l0, const LevelDesc& lf, const LevelDesc* lc,
                             const double* tf, const double* tc, int n, double* y, double* y2,
                             unsigned long long* cens, cudaStream_t st) {
  int64_t total = (int64_t)n * l0.nodes;
  if (total == 0) return cudaSuccess;
  int bs = 256;
  pair_diff_kernel<<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>(
      l0, lf, lc ? *lc : l0, lc != nullptr, tf, tc, n, y, y2, cens);
  return cudaGetLastError();
}

// One thread per coarsest-grid node; the batch is read in sample order.
__global__ void accumulate_kernel(int64_t nodes0, const double* __restrict__ y,
                                  const double* __restrict__ y2, int n, int64_t n_old,
                                  double* __restrict__ mean, double* __restrict__ m2,
                                  double* __restrict__ mean2) {
  int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (A >= nodes0 || n == 0) return;
  double sb = 0.0, sb2 = 0.0;
  for (int s = 0; s < n; ++s) {
    sb += y[(int64_t)s * nodes0 + A];
    sb2 += y2[(int64_t)s * nodes0 + A];
  }
  double mb = sb / n, mb2 = sb2 / n;
  double M2b = 0.0;
  for (int s = 0; s < n; ++s) {
    double dv = y[(int64_t)s * nodes0 + A] - mb;
    M2b += dv * dv;
  }
  double na = (double)n_old, nb = (double)n, nt = na + nb;
  double ma = mean[A], ma2 = mean2[A];
  double delta = mb - ma;
  mean[A] = ma + delta * nb / nt;
  m2[A] = m2[A] + M2b + delta * delta * na * nb / nt;
  mean2[A] = ma2 + (mb2 - ma2) * nb / nt;
}

cudaError_t launch_accumulate(int64_t nodes0, const double* y, const double* y2, int n,
                              int64_t n_old, double* mean, double* m2, double* mean2,
                              cudaStream_t st) {
  if (n == 0 || nodes0 == 0) return cudaSuccess;
  int bs = 128;
  accumulate_kernel<<<(unsigned)((nodes0 + bs - 1) / bs), bs, 0, st>>>(nodes0, y, y2, n, n_old,
                                                                        mean, m2, mean2);
  return cudaGetLastError();
}

// Single block.  out = [mean | var | mean_l (L x n0) | var_l (L x n0) | V_l (L) | bias | rmse].
__global__ void estimate_kernel(int L, int64_t n0, LevelDesc l0, const int64_t* __restrict__ N_l,
                                const double* __restrict__ mean_l, const double* __restrict__ m2_l,
                                const double* __restrict__ mean2_l, double* __restrict__ out) {
  __shared__ double red[32];
  double* mean = out;
  double* var = out + n0;
  double* o_mean_l = out + 2 * n0;
  double* o_var_l = o_mean_l + (int64_t)L * n0;
  double* V = o_var_l + (int64_t)L * n0;
  double* tail = V + L;  // bias, rmse
  double vloc[MLMC_MAX_LEVELS];
  for (int l = 0; l < L; ++l) vloc[l] = 0.0;
  double bias_loc = 0.0;
  for (int64_t A = threadIdx.x; A < n0; A += blockDim.x) {
    int i, j, k;
    node_ijk(l0, A, i, j, k);
    double w = lumped_mass(l0, i, j, k);
    double mu = 0.0, e2 = 0.0;
    for (int l = 0; l < L; ++l) {
      double ml = mean_l[(int64_t)l * n0 + A];
      double vl = N_l[l] > 1 ? m2_l[(int64_t)l * n0 + A] / (double)(N_l[l] - 1) : 0.0;
      o_mean_l[(int64_t)l * n0 + A] = ml;
      o_var_l[(int64_t)l * n0 + A] = vl;
      vloc[l] += w * vl;
      mu += ml;
      e2 += mean2_l[(int64_t)l * n0 + A];
    }
    mean[A] = mu;
    var[A] = fmax(e2 - mu * mu, 0.0);
    if (L > 1) {
      double mL = mean_l[(int64_t)(L - 1) * n0 + A];
      bias_loc += w * mL * mL;
    }
  }
  // fixed-order block reductions of V_l and the bias
  for (int l = 0; l <= L; ++l) {
    double v = l < L ? vloc[l] : bias_loc;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      if (l < L) V[l] = t; else tail[0] = sqrt(t);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double r2 = tail[0] * tail[0];
    for (int l = 0; l < L; ++l) r2 += N_l[l] > 0 ? V[l] / (double)N_l[l] : 0.0;
    tail[1] = sqrt(r2);
  }
}

cudaError_t launch_estimate(int levels, int64_t nodes0, const LevelDesc& l0, const int64_t* N_l,
                            const double* mean_l, const double* m2_l, const double* mean2_l,
                            double* out, cudaStream_t st) {
  estimate_kernel<<<1, 256, 0, st>>>(levels, nodes0, l0, N_l, mean_l, m2_l, mean2_l, out);
  return cudaGetLastError();
}

}  // namespace mlmc
