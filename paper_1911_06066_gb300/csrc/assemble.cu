// Row a3: per-sample conductivity and Q1 stiffness couplings (Sec. 3.2,
// Eq. semi-disc: K = [int (G grad psi_i) . grad psi_j]), with the cell-constant
// fiber tensor D = s_t I + (s_l - s_t) f f^T, s_l = s_l0 exp(Z),
// f = (cos th, sin th, 0), th = theta0 in 2D and linear in the centroid's z in 3D.
//
// Element matrix of a box with sides (hx, hy[, hz]) and constant D, integrated
// exactly: with s(b) = -1/+1 for local coordinate 0/1 and the 1D mass weights
// m1(p,q) = 1/3 (p == q) or 1/6 (p != q) on the unit interval,
//   2D: K_ab = Dxx sx_a sx_b (hy/hx) m1(ay,by) + Dyy sy_a sy_b (hx/hy) m1(ax,bx)
//            + Dxy (sx_a sy_b + sy_a sx_b) / 4
//   3D: K_ab = Dxx sx_a sx_b (hy hz/hx) m1(ay,by) m1(az,bz) + (y, z analogues)
//            + Dxy (sx_a sy_b + sy_a sx_b) hz m1(az,bz) / 4 + (xz, yz analogues).
// Each node gathers the rows of the 2^dim cells around it into its 3^dim
// couplings, stored [sample][offset][node] (offset (dx,dy,dz) in {-1,0,1}^dim,
// x fastest), so no two threads write the same entry; or, for the 3D
// global-memory sweeps (sym), only the offsets 13..26 (see launch_assemble).
#include <math.h>

#include "internal.cuh"

namespace mlmc {

__device__ inline double m1(int p, int q) { return p == q ? (1.0 / 3.0) : (1.0 / 6.0); }
__device__ inline double sgn(int b) { return b ? 1.0 : -1.0; }

__device__ double element_entry(int dim, const double D[3][3], const double h[3], const int a[3],
                                const int b[3]) {
  if (dim == 1) return D[0][0] * sgn(a[0]) * sgn(b[0]) / h[0];
  if (dim == 2) {
    return D[0][0] * sgn(a[0]) * sgn(b[0]) * (h[1] / h[0]) * m1(a[1], b[1]) +
           D[1][1] * sgn(a[1]) * sgn(b[1]) * (h[0] / h[1]) * m1(a[0], b[0]) +
           D[0][1] * (sgn(a[0]) * sgn(b[1]) + sgn(a[1]) * sgn(b[0])) * 0.25;
  }
  double k = 0.0;
  for (int p = 0; p < 3; ++p) {
    int q1 = (p + 1) % 3, q2 = (p + 2) % 3;
    k += D[p][p] * sgn(a[p]) * sgn(b[p]) * (h[q1] * h[q2] / h[p]) * m1(a[q1], b[q1]) * m1(a[q2], b[q2]);
  }
  for (int p = 0; p < 3; ++p)
    for (int q = p + 1; q < 3; ++q) {
      int r = 3 - p - q;
      k += D[p][q] * (sgn(a[p]) * sgn(b[q]) + sgn(a[q]) * sgn(b[p])) * h[r] * m1(a[r], b[r]) * 0.25;
    }
  return k;
}

template <int DIM>
__global__ void assemble_kernel(LevelDesc lv, Physics ph, const double* __restrict__ Z, int n,
                                double* __restrict__ coef64, float* __restrict__ coef32, int sym) {
  constexpr int NO = DIM == 3 ? 27 : (DIM == 2 ? 9 : 3);
  constexpr int CTR = NO / 2;
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)n * lv.nodes) return;
  int s = (int)(g / lv.nodes);
  int64_t A = g % lv.nodes;
  int ijk[3];
  node_ijk(lv, A, ijk[0], ijk[1], ijk[2]);
  double K[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) K[o] = 0.0;
  const double* Zs = Z + (int64_t)s * lv.cells;
  for (int cz = (DIM == 3 ? -1 : 0); cz <= 0; ++cz)
    for (int cy = (DIM >= 2 ? -1 : 0); cy <= 0; ++cy)
      for (int cx = -1; cx <= 0; ++cx) {
        int cell[3] = {ijk[0] + cx, ijk[1] + cy, ijk[2] + cz};
        bool ok = true;
        for (int d = 0; d < DIM; ++d) ok = ok && cell[d] >= 0 && cell[d] < lv.n[d];
        if (!ok) continue;
        int64_t ci = ((int64_t)cell[2] * lv.n[1] + cell[1]) * lv.n[0] + cell[0];
        double th = ph.th0;
        if (DIM == 3) th = ph.th0 + (ph.th1 - ph.th0) * ((cell[2] + 0.5) * lv.h[2]) / ph.Lz;
        double f[3] = {cos(th), sin(th), 0.0};
        double D[3][3];
        if (ph.cond_kind == 1) {   // the paper's isotropic G = G0 (1 + Z)
          const double g = ph.s_l0 * (1.0 + Zs[ci]);
          for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) D[p][q] = p == q ? g : 0.0;
        } else {
          const double sl = ph.s_l0 * exp(Zs[ci]);
          for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) D[p][q] = (p == q ? ph.s_t : 0.0) + (sl - ph.s_t) * f[p] * f[q];
        }
        int a[3] = {-cx, -cy, -cz};
        for (int bz = 0; bz < (DIM == 3 ? 2 : 1); ++bz)
          for (int by = 0; by < (DIM >= 2 ? 2 : 1); ++by)
            for (int bx = 0; bx < 2; ++bx) {
              int b[3] = {bx, by, bz};
              int o = (bx - a[0] + 1) + (DIM >= 2 ? 3 * (by - a[1] + 1) : 0) +
                      (DIM == 3 ? 9 * (bz - a[2] + 1) : 0);
              K[o] += element_entry(DIM, D, lv.h, a, b);
            }
      }
  // stored times theta (1 implicit Euler, 1/2 Crank-Nicolson): the Hessian's
  // stiffness part, and with (1-theta)/theta the explicit part of the residual
  // with sym only the offsets CTR..NO-1 are stored, at CTR..NO-1 minus CTR
  const int nst = sym ? NO - CTR : NO;
  int64_t base = (int64_t)s * nst * lv.nodes + A;
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    if (sym && o < CTR) continue;
    const int oi = sym ? o - CTR : o;
    const double k = ph.theta * K[o];
    coef64[base + (int64_t)oi * lv.nodes] = k;
    if (coef32) coef32[base + (int64_t)oi * lv.nodes] = (float)k;
  }
}

cudaError_t launch_assemble(const LevelDesc& lv, const Physics& ph, const double* Z, int n,
                            double* coef64, float* coef32, cudaStream_t st, bool sym) {
  int64_t total = (int64_t)n * lv.nodes;
  if (total == 0) return cudaSuccess;
  if (sym && lv.dim != 3) return cudaErrorInvalidValue;
  int bs = 128;
  unsigned grid = (unsigned)((total + bs - 1) / bs);
  if (lv.dim == 3)
    assemble_kernel<3><<<grid, bs, 0, st>>>(lv, ph, Z, n, coef64, coef32, sym ? 1 : 0);
  else if (lv.dim == 2)
    assemble_kernel<2><<<grid, bs, 0, st>>>(lv, ph, Z, n, coef64, coef32, 0);
  else
    assemble_kernel<1><<<grid, bs, 0, st>>>(lv, ph, Z, n, coef64, coef32, 0);
  return cudaGetLastError();
}

cudaError_t preload_assemble() {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, assemble_kernel<2>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, assemble_kernel<1>);
  return e == cudaSuccess ? cudaFuncGetAttributes(&a, assemble_kernel<3>) : e;
}

}  // namespace mlmc
