// Rows a4-a8: the per-sample nonlinear space-time solve (Sec. 3.3, Eq. mono_disc,
// in the implicit-Euler variant; Sec. 3.5: Newton).
//
// The space-time system is block lower-bidiagonal in time (Sec. 3.2,
// Eq. system_C), so Newton's linear systems are solved by forward block
// substitution, and this kernel sweeps the slab forward: block row k,
//   F_k(u) = (M/dt)(u_k - u_{k-1}) + K u_k - M r(u_k),  r(u) = c u(1-u)(u-a),
// is driven to convergence from the initial guess u_{k-1} before row k+1.
// Its Jacobian block H = M/dt + K - M diag(r'(u)) is symmetric -- F_k is the
// gradient of the step energy
//   E(u) = (u-u_{k-1})^T M (u-u_{k-1})/(2dt) + u^T K u/2 - sum_i M_i R(u_i),  R' = r
// -- and indefinite when c dt max r' > 1, where the step has several roots
// (local minima of E).  The root is the end point of the gradient flow
// M v' = -F_k(v) from u_{k-1}: the minimum in whose basin u_{k-1} lies.
//   * Levels with several roots (sp.flow): gradient-flow continuation by
//     linearly implicit pseudo-steps (M/t + H(u)) d = -F(u), u += d, with the
//     pseudo-step t from 1/(2 max r') growing towards a move limit (at most
//     x2 per step), retried with t/4 when the CG meets non-positive curvature
//     (M/t + H must stay positive definite), taken shortened when it would
//     move a node by more than FLOW_MOVE, and finished by Newton steps (t =
//     infinity) once the flow has nearly arrived (see SolverParams in
//     internal.cuh).
//   * Other levels: H is positive definite for every state and the root
//     unique; Newton with Armijo backtracking on E (sigma = 1e-4, halving, at
//     most 40; the energy change summed node by node in a cancellation-free
//     form; full step when max|d| <= ls_full_step).
//   * Linear solves by CG with the Jacobi preconditioner |diag|, from 0,
//     until the preconditioned residual drops by lin_rtol; truncated at the
//     first direction with p^T A p <= 0 (then the current iterate, or the
//     preconditioned steepest-descent step in the first iteration).
//   * Stop once an accepted step moves no node by more than newton_tol.
//
// GPU mapping: one thread block per sample; every block loops over all time
// steps, Newton and CG iterations on its own, so the whole slab of a batch is
// one launch with no grid-wide synchronisation.  Vectors live in the per-sample
// workspace (L2-resident at these sizes); dot products are block reductions in
// a fixed order (warp butterflies, then warps in index order), so results are
// deterministic.  KR is the type of the CG vectors and stencil copy: double for
// the FP64 path, float for the mixed path (residual, update, line search and
// activation stay FP64 in both).  Activation times (row a8: first crossing of
// 1/2, linear in t) are extracted on the fly.
#include <math.h>

#include "internal.cuh"

namespace mlmc {

constexpr int SOLVE_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the block in a fixed order; every thread gets the result.
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < SOLVE_THREADS / 32; ++w) t += sh[w];
  __syncthreads();
  return t;
}
__device__ double block_max(double v, double* sh) {
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < SOLVE_THREADS / 32; ++w) t = fmax(t, sh[w]);
  __syncthreads();
  return t;
}

template <int DIM>
__device__ __forceinline__ int64_t nb_offset(const LevelDesc& lv, int o) {
  int dx = o % 3 - 1, dy = (DIM >= 2 ? (o / 3) % 3 - 1 : 0), dz = DIM == 3 ? o / 9 - 1 : 0;
  return dx + (int64_t)lv.N[0] * (dy + (int64_t)lv.N[1] * dz);
}

// (K v)_A from the node's couplings; out-of-domain couplings are zero, so the
// neighbour index only has to stay inside the array.
template <int DIM, typename TC, typename TV, typename TA>
__device__ __forceinline__ TA stencil(const LevelDesc& lv, const TC* __restrict__ c,
                                      const TV* __restrict__ v, int64_t A) {
  constexpr int NO = DIM == 3 ? 27 : (DIM == 2 ? 9 : 3);
  TA y = 0;
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    int64_t B = A + nb_offset<DIM>(lv, o);
    B = B < 0 ? 0 : (B >= lv.nodes ? lv.nodes - 1 : B);
    y += (TA)c[(int64_t)o * lv.nodes + A] * (TA)v[B];
  }
  return y;
}

template <typename KR, int DIM>
__global__ void __launch_bounds__(SOLVE_THREADS)
solve_kernel(LevelDesc lv, Physics ph, SolverParams sp, const double* __restrict__ coef64,
             const KR* __restrict__ coefK, double* slab, double* ubuf, double* Fb, double* Kub,
             double* Kdb, KR* krb, double* t_act, mlmc_sample_info* info,
             unsigned long long* counters) {
  constexpr int NO = DIM == 3 ? 27 : (DIM == 2 ? 9 : 3);
  __shared__ double sh[SOLVE_THREADS / 32];
  const int s = blockIdx.x;
  const int64_t N = lv.nodes;
  const double* c64 = coef64 + (int64_t)s * NO * N;
  const KR* cK = coefK + (int64_t)s * NO * N;
  double* F = Fb + (int64_t)s * N;
  double* Ku = Kub + (int64_t)s * N;
  double* Kd = Kdb + (int64_t)s * N;
  KR* r = krb + (int64_t)s * 7 * N;
  KR* z = r + N;
  KR* p = z + N;
  KR* q = p + N;
  KR* d = q + N;
  KR* hm = d + N;
  KR* pinv = hm + N;
  double* ta = t_act + (int64_t)s * N;
  double* sl = slab ? slab + (int64_t)s * (lv.m + 1) * N : nullptr;
  double* ub = ubuf + (int64_t)s * 2 * N;
  const double dt = lv.dt, inv_dt = 1.0 / lv.dt;

  // initial state: the stimulus ball; activation 0 where already >= 1/2
  double* u0 = sl ? sl : ub;
  double sc[3];
  for (int dd = 0; dd < 3; ++dd) sc[dd] = ph.stim_ps ? ph.stim_ps[3 * s + dd] : ph.stim_c[dd];
  for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) {
    int i, j, k;
    node_ijk(lv, A, i, j, k);
    double x[3] = {i * lv.h[0], j * lv.h[1], k * lv.h[2]};
    double r2 = 0.0;
    for (int dd = 0; dd < DIM; ++dd) r2 += (x[dd] - sc[dd]) * (x[dd] - sc[dd]);
    double v = ph.stim_kind == 0 && r2 < ph.stim_r2 ? 1.0 : 0.0;
    u0[A] = v;
    ta[A] = v >= 0.5 ? 0.0 : -1.0;
  }
  __syncthreads();

  int status = MLMC_OK, failed_step = 0;
  int newton_total = 0, cg_total = 0, trunc_total = 0, halvings = 0, max_newton = 0;
  for (int step = 1; step <= lv.m; ++step) {
    const double* up = sl ? sl + (int64_t)(step - 1) * N : ub + (int64_t)((step - 1) & 1) * N;
    double* u = sl ? sl + (int64_t)step * N : ub + (int64_t)(step & 1) * N;
    // start: u_{k-1}, or on levels with a unique root (no continuation) the
    // linear extrapolation 2 u_{k-1} - u_{k-2}, which the root does not depend on
    const double* upp = step < 2 || sp.flow ? nullptr
                        : (sl ? sl + (int64_t)(step - 2) * N : u);   // u still holds u_{k-2}
    for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) u[A] = upp ? 2.0 * up[A] - upp[A] : up[A];
    __syncthreads();
    const double c_up = (1.0 - ph.theta) / ph.theta;      // Crank-Nicolson: explicit part
    const double src_scale = stim_step_scale(ph, step, dt);
    double tau = sp.tau0, sw = FLOW_NEWTON;
    bool newton_phase = false;
    bool conv = false, lin_fail = false;
    int it;
    for (it = 1; it <= sp.newton_max; ++it) {
      const double t = tau;
      const double shift = sp.flow && !newton_phase ? 1.0 / t : 0.0;
      // residual, Hessian diagonal, CG start (r = -F, z = P^-1 r, p = z, d = 0).
      // FP32 CG on grids with a tiny lumped mass per time step (sp.cg_scale):
      // the right-hand side is scaled by the power of two sigma with
      // ||F||_2 sigma in [1, 2) and d by 1/sigma after the solve (exact), so
      // that the CG's products stay in FP32's normal range.
      const bool SCALE = sizeof(KR) == 4 && sp.cg_scale != 0;
      double rz_loc = 0.0, f2_loc = 0.0;
      for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) {
        int i, j, k;
        node_ijk(lv, A, i, j, k);
        double mA = lumped_mass(lv, i, j, k);
        double uA = u[A];
        // Ku: the part of the residual linear in u and the explicit terms
        // (theta K u + (1-theta) K u_{k-1} - M s_k); the energy line search
        // uses it as the linear coefficient of its step length
        double ku = stencil<DIM, double, double, double>(lv, c64, u, A);
        if (c_up != 0.0) ku += c_up * stencil<DIM, double, double, double>(lv, c64, up, A);
        if (src_scale != 0.0) ku -= mA * src_scale * stim_shape(ph, lv, sc, i, j, k);
        Ku[A] = ku;
        double f = ku + mA * inv_dt * (uA - up[A]) - mA * rxn(ph, uA);
        F[A] = f;
        double hmA = mA * (inv_dt + shift) - mA * rxn_d(ph, uA);
        double pv = 1.0 / fabs(hmA + c64[(int64_t)centre_offset(DIM) * N + A]);
        KR rv = (KR)(-f);
        KR zv = (KR)pv * rv;
        hm[A] = (KR)hmA;
        pinv[A] = (KR)pv;
        r[A] = rv; z[A] = zv; p[A] = zv; d[A] = (KR)0;
        rz_loc += (double)(rv * zv);
        f2_loc += f * f;
      }
      double sigma = 1.0;
      if (SCALE) {
        const double f2 = block_sum(f2_loc, sh);
        if (f2 > 0.0) sigma = ldexp(1.0, -ilogb(sqrt(f2)));
        rz_loc = 0.0;
        for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) {
          const KR rv = (KR)(-F[A] * sigma);
          const KR zv = pinv[A] * rv;
          r[A] = rv; z[A] = zv; p[A] = zv;
          rz_loc += (double)(rv * zv);
        }
      }
      double rz = block_sum(rz_loc, sh);
      const double r0 = sqrt(rz);
      int cg = 0;
      bool truncated = false;
      if (r0 > 0.0) {
        bool ok = false;
        for (cg = 1; cg <= sp.lin_max; ++cg) {
          KR pq_loc = 0;
          for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) {
            KR qv = stencil<DIM, KR, KR, KR>(lv, cK, p, A) + hm[A] * p[A];
            q[A] = qv;
            pq_loc += p[A] * qv;
          }
          double pq = block_sum((double)pq_loc, sh);
          if (pq <= 0.0) {
            truncated = true;
            if (cg == 1)
              for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) d[A] = z[A];
            ok = true;
            break;
          }
          const KR alpha = (KR)(rz / pq);
          KR rz_new_loc = 0;
          for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) {
            d[A] += alpha * p[A];
            KR rv = r[A] - alpha * q[A];
            KR zv = pinv[A] * rv;
            r[A] = rv;
            z[A] = zv;
            rz_new_loc += rv * zv;
          }
          double rz_new = block_sum((double)rz_new_loc, sh);
          if (sqrt(rz_new) <= sp.lin_rtol * r0) { ok = true; break; }
          const KR beta = (KR)(rz_new / rz);
          for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) p[A] = z[A] + beta * p[A];
          __syncthreads();
          rz = rz_new;
        }
        if (!ok) { lin_fail = true; cg = sp.lin_max; }
      }
      cg_total += cg;
      trunc_total += truncated ? 1 : 0;
      if (lin_fail) break;
      if (SCALE && sigma != 1.0) {
        const KR inv_sigma = (KR)(1.0 / sigma);   // a power of two: exact
        for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) d[A] *= inv_sigma;
        __syncthreads();
      }
      double dmax_loc = 0.0;
      for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) dmax_loc = fmax(dmax_loc, fabs((double)d[A]));
      const double dmax = block_max(dmax_loc, sh);
      if (sp.flow) {
        bool accept;
        if (newton_phase) {
          accept = !(truncated || dmax > 10.0 * sw);
          if (!accept) { newton_phase = false; sw *= 0.1; ++halvings; }
        } else if (truncated && t > FLOW_TMIN) {
          accept = false;              // M/t + H not positive definite
          tau = 0.25 * t;
          ++halvings;
        } else {
          accept = true;
        }
        if (!accept) continue;       // the state is unchanged; retry
        if (!newton_phase && dmax > FLOW_MOVE && t > FLOW_TMIN) {
          // the step would move a node by more than FLOW_MOVE: take it
          // shortened to that move (a positive multiple keeps its sign along
          // every eigenvector of M/t + H); the next pseudo-step is shorter
          const double sc = FLOW_MOVE / dmax;
          for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) u[A] += sc * (double)d[A];
          __syncthreads();
          tau = t * 0.9 * sc;
          ++halvings;
          continue;
        }
        for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) u[A] += (double)d[A];
        __syncthreads();
        if (dmax <= sp.newton_tol) { conv = true; break; }
        if (!newton_phase) {
          if (dmax <= sw) newton_phase = true;
          tau = fmin(t * fmin(2.0, 0.9 * FLOW_MOVE / dmax), FLOW_TMAX);   // towards the move limit
        }
        continue;
      }
      double alpha = 1.0;
      if (dmax > sp.newton_tol && dmax > sp.ls_full_step) {
        double gd_loc = 0.0;
        for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) {
          Kd[A] = stencil<DIM, double, KR, double>(lv, c64, d, A);
          gd_loc += F[A] * (double)d[A];
        }
        const double gd = block_sum(gd_loc, sh);
        for (int h = 0; h < 40; ++h) {
          double e_loc = 0.0;
          for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) {
            int i, j, k;
            node_ijk(lv, A, i, j, k);
            double mA = lumped_mass(lv, i, j, k);
            double uA = u[A], w = alpha * (double)d[A], v = uA + w;
            double sm = v + uA, q2 = v * v + uA * uA, q3 = v * v + v * uA + uA * uA;
            double rdiff = ph.c * w * (-sm * q2 / 4.0 + (1.0 + ph.a) * q3 / 3.0 - ph.a * sm / 2.0);
            e_loc += mA * w * (2.0 * (uA - up[A]) + w) / (2.0 * dt) + w * Ku[A] +
                     0.5 * w * alpha * Kd[A] - mA * rdiff;
          }
          double dE = block_sum(e_loc, sh);
          if (dE <= 1e-4 * alpha * gd) break;
          alpha *= 0.5;
          ++halvings;
        }
      }
      for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) u[A] += alpha * (double)d[A];
      __syncthreads();
      if (dmax <= sp.newton_tol) { conv = true; break; }
    }
    int used = it > sp.newton_max ? sp.newton_max : it;
    newton_total += used;
    max_newton = used > max_newton ? used : max_newton;
    if (!conv) { status = MLMC_ERR_NOT_CONVERGED; failed_step = step; break; }
    for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) {
      if (ta[A] < 0.0 && u[A] >= 0.5) {
        double uo = up[A];
        ta[A] = (double)(step - 1) * dt + dt * (0.5 - uo) / (u[A] - uo);
      }
    }
    // the next step reads u as up after the sync at its start
  }
  {
    // the quantity of interest: activation times (T where never reached), or
    // the final state u(T)
    const double* ufin = sl ? sl + (int64_t)lv.m * N : ub + (int64_t)(lv.m & 1) * N;
    for (int64_t A = threadIdx.x; A < N; A += SOLVE_THREADS) {
      if (ph.qoi == 1) ta[A] = ufin[A];
      else if (ta[A] < 0.0) ta[A] = lv.T;
    }
  }
  if (counters && threadIdx.x == 0) {
    if (status != MLMC_OK) atomicAdd(counters, 1ull);
    atomicAdd(counters + 1, (unsigned long long)cg_total * (unsigned long long)N);
    atomicAdd(counters + 2, (unsigned long long)newton_total * (unsigned long long)N);
    atomicAdd(counters + 3, (unsigned long long)trunc_total);
    atomicAdd(counters + 4, (unsigned long long)halvings);
    if (sizeof(KR) == 8) atomicAdd(counters + 5, (unsigned long long)cg_total * (unsigned long long)N);
  }
  if (info && threadIdx.x == 0) {
    mlmc_sample_info o;
    o.status = status; o.failed_step = failed_step; o.newton_iters = newton_total;
    o.cg_iters = cg_total; o.truncations = trunc_total; o.halvings = halvings;
    o.max_newton = max_newton; o.pad = 0;
    info[s] = o;
  }
}

cudaError_t launch_solve(const LevelDesc& lv, const Physics& ph, const SolverParams& sp,
                         bool mixed, int n, const double* coef64, const float* coef32,
                         double* slab, double* ubuf, double* F, double* Ku, double* Kd,
                         void* kr, double* t_act, mlmc_sample_info* info,
                         unsigned long long* counters, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
#define SOLVE_LAUNCH(KR, D, CK)                                                                  \
  solve_kernel<KR, D><<<n, SOLVE_THREADS, 0, st>>>(lv, ph, sp, coef64, CK, slab, ubuf, F, Ku, Kd,  \
                                                  (KR*)kr, t_act, info, counters)
  if (mixed) {
    if (lv.dim == 3) SOLVE_LAUNCH(float, 3, coef32);
    else if (lv.dim == 2) SOLVE_LAUNCH(float, 2, coef32);
    else SOLVE_LAUNCH(float, 1, coef32);
  } else {
    if (lv.dim == 3) SOLVE_LAUNCH(double, 3, coef64);
    else if (lv.dim == 2) SOLVE_LAUNCH(double, 2, coef64);
    else SOLVE_LAUNCH(double, 1, coef64);
  }
#undef SOLVE_LAUNCH
  return cudaGetLastError();
}

cudaError_t preload_solve(const LevelDesc& lv, bool mixed) {
  cudaFuncAttributes a;
  if (mixed)
    return lv.dim == 3   ? cudaFuncGetAttributes(&a, solve_kernel<float, 3>)
           : lv.dim == 2 ? cudaFuncGetAttributes(&a, solve_kernel<float, 2>)
                         : cudaFuncGetAttributes(&a, solve_kernel<float, 1>);
  return lv.dim == 3   ? cudaFuncGetAttributes(&a, solve_kernel<double, 3>)
         : lv.dim == 2 ? cudaFuncGetAttributes(&a, solve_kernel<double, 2>)
                       : cudaFuncGetAttributes(&a, solve_kernel<double, 1>);
}

}  // namespace mlmc
