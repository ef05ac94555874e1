// Row a4 over the whole slab and row a8 from a stored slab.
//
// slab_residual: the all-at-once space-time residual (Sec. 3.3, Eq. mono_disc
// with the blocks of Eq. system_C: implicit Euler or Crank-Nicolson, Sec. 3.2),
// every (sample, slice, node) in one launch:
//   F[s][k-1][A] = (K (theta u_k + (1-theta) u_{k-1}))_A + (M_A/dt)(u_k - u_{k-1})_A
//                  - M_A r(u_k,A) - M_A s_k,A,  k = 1..m,
// and res_max[s] = max |F| / M_A, the convergence certificate of the slab.
// Memory-bound stream: reads u_k, u_{k-1} (the latter from L2/L1 when adjacent
// slices are processed by neighbouring blocks) and the couplings, writes F.
//
// activation: first crossing of 1/2 per node, linear in time; 0 where
// u_0 >= 1/2, T where never crossed.
#include <math.h>

#include "internal.cuh"

namespace mlmc {

template <int DIM>
__global__ void slab_residual_kernel(LevelDesc lv, Physics ph, const double* __restrict__ coef64,
                                     const double* __restrict__ slab, double* __restrict__ F,
                                     unsigned long long* __restrict__ res_max) {
  constexpr int NO = DIM == 3 ? 27 : (DIM == 2 ? 9 : 3);
  __shared__ double wmax[32];
  const int64_t N = lv.nodes;
  const int s = blockIdx.y;                       // one sample per grid row
  const int64_t per_sample = (int64_t)lv.m * N;
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double rel = 0.0;
  if (g < per_sample) {
    int k = (int)(g / N) + 1;
    int64_t A = g % N;
    const double* u = slab + ((int64_t)s * (lv.m + 1) + k) * N;
    const double* up = u - N;
    const double* c = coef64 + (int64_t)s * NO * N;
    double ku = 0.0;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      int dx = o % 3 - 1, dy = (DIM >= 2 ? (o / 3) % 3 - 1 : 0), dz = DIM == 3 ? o / 9 - 1 : 0;
      int64_t B = A + dx + (int64_t)lv.N[0] * (dy + (int64_t)lv.N[1] * dz);
      B = B < 0 ? 0 : (B >= N ? N - 1 : B);
      ku += c[(int64_t)o * N + A] * u[B];
    }
    // Crank-Nicolson: (1-theta)/theta times the theta-scaled stencil of u_{k-1}
    const double c_up = (1.0 - ph.theta) / ph.theta;
    if (c_up != 0.0) {
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        int dx = o % 3 - 1, dy = (DIM >= 2 ? (o / 3) % 3 - 1 : 0), dz = DIM == 3 ? o / 9 - 1 : 0;
        int64_t B = A + dx + (int64_t)lv.N[0] * (dy + (int64_t)lv.N[1] * dz);
        B = B < 0 ? 0 : (B >= N ? N - 1 : B);
        ku += c_up * c[(int64_t)o * N + A] * up[B];
      }
    }
    int i, j, kk;
    node_ijk(lv, A, i, j, kk);
    double mA = lumped_mass(lv, i, j, kk);
    double uA = u[A];
    double f = ku + mA / lv.dt * (uA - up[A]) - mA * rxn(ph, uA);
    const double src = stim_step_scale(ph, k, lv.dt);
    if (src != 0.0) {
      double sc[3];
      for (int d = 0; d < 3; ++d) sc[d] = ph.stim_ps ? ph.stim_ps[3 * s + d] : ph.stim_c[d];
      f -= mA * src * stim_shape(ph, lv, sc, i, j, kk);
    }
    if (F) F[(int64_t)s * per_sample + g] = f;
    rel = fabs(f) / mA;
  }
  if (res_max) {
    // block max, then one atomic per block (non-negative doubles order like
    // their bit patterns)
    for (int o = 16; o > 0; o >>= 1) rel = fmax(rel, __shfl_xor_sync(0xffffffffu, rel, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = rel;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wmax[w]);
      atomicMax(res_max + s, (unsigned long long)__double_as_longlong(m));
    }
  }
}

cudaError_t launch_slab_residual(const LevelDesc& lv, const Physics& ph, const double* coef64,
                                 const double* slab, int n, double* F, double* res_max,
                                 cudaStream_t st) {
  int64_t per_sample = (int64_t)lv.m * lv.nodes;
  if (res_max) {
    cudaError_t e = cudaMemsetAsync(res_max, 0, sizeof(double) * n, st);
    if (e != cudaSuccess) return e;
  }
  if (n == 0 || per_sample == 0) return cudaSuccess;
  int bs = 256;
  dim3 grid((unsigned)((per_sample + bs - 1) / bs), (unsigned)n);
  if (lv.dim == 3)
    slab_residual_kernel<3><<<grid, bs, 0, st>>>(lv, ph, coef64, slab, F, (unsigned long long*)res_max);
  else if (lv.dim == 2)
    slab_residual_kernel<2><<<grid, bs, 0, st>>>(lv, ph, coef64, slab, F, (unsigned long long*)res_max);
  else
    slab_residual_kernel<1><<<grid, bs, 0, st>>>(lv, ph, coef64, slab, F, (unsigned long long*)res_max);
  return cudaGetLastError();
}

__global__ void activation_kernel(LevelDesc lv, const double* __restrict__ slab, int n,
                                  double* __restrict__ t_act) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)n * lv.nodes) return;
  int s = (int)(g / lv.nodes);
  int64_t A = g % lv.nodes;
  const double* u = slab + (int64_t)s * (lv.m + 1) * lv.nodes + A;
  double t = lv.T;
  if (u[0] >= 0.5) {
    t = 0.0;
  } else {
    for (int k = 1; k <= lv.m; ++k) {
      double uk = u[(int64_t)k * lv.nodes];
      if (uk >= 0.5) {
        double uo = u[(int64_t)(k - 1) * lv.nodes];
        t = (double)(k - 1) * lv.dt + lv.dt * (0.5 - uo) / (uk - uo);
        break;
      }
    }
  }
  t_act[g] = t;
}

cudaError_t launch_activation(const LevelDesc& lv, const double* slab, int n, double* t_act,
                              cudaStream_t st) {
  int64_t total = (int64_t)n * lv.nodes;
  if (total == 0) return cudaSuccess;
  int bs = 256;
  activation_kernel<<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>(lv, slab, n, t_act);
  return cudaGetLastError();
}

}  // namespace mlmc
