/*
 * Oracle: the nonlinear space-time problem of one sample (Sec. 3.3,
 * Eq. mono_disc) in the implicit-Euler variant, solved step by step.
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * Block row k of the space-time system (k = 1..m, dt = T/m, M lumped):
 *   F_k(u) = (M/dt)(u_k - u_{k-1}) + K u_k - M r(u_k),   r(u) = c u (1-u)(u-a)
 * (the FHN current of Eq. ionic_term written as -c u(1-u)(u-a) on [0,1]).
 * Its Jacobian block (Sec. 3.3) is  H = M/dt + K - M diag(r'(u)),
 *   r'(u) = c(-3u^2 + 2(1+a)u - a).
 * H is symmetric, so F_k is the gradient of the step energy
 *   E(u) = (u-u_{k-1})^T M (u-u_{k-1}) / (2dt) + u^T K u / 2 - sum_i m_i R(u_i),
 *   R' = r,
 * and H is its Hessian.  When c dt max r' > 1 the step has several roots and
 * plain Newton from u_{k-1} cycles, so the root is defined (the paper is
 * silent) as the one reached from u_{k-1} by line-search Newton-CG on E
 * (Nocedal & Wright, Numerical Optimization, Alg. 7.1):
 *   - d from Jacobi-preconditioned CG (preconditioner |diag H|) on H d = -F,
 *     started at 0, stopped at relative preconditioned residual lin_rtol, and
 *     truncated at the first search direction p with p^T H p <= 0 (then the
 *     current iterate, or the preconditioned steepest-descent step if that
 *     happens in the first iteration);
 *   - stop when max|d| <= newton_tol (after applying d);
 *   - on strongly indefinite steps (c dt max r' > 2, max r' = c((1+a)^2/3 - a))
 *     the step starts at alpha = min(1, 0.1 / max|d|): no node moves by more
 *     than 0.1 per iteration, so the iterates follow the descent path instead
 *     of jumping between basins of attraction, which makes the selected root
 *     insensitive to rounding (with full steps, perturbations of one ulp in the
 *     couplings changed the root in 8 of 16 samples of a 3D level);
 *   - otherwise Armijo backtracking (halving, sigma = 1e-4, at most 40 halvings)
 *     on E(u + alpha d) - E(u) <= sigma alpha F^T d, with the energy change
 *     summed node by node in a cancellation-free form; when max|d| <= 1e-6 the
 *     full step is taken (the energy change is then below round-off).
 * Where H is positive definite this is plain Newton with full steps.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static double rxn(double c, double a, double u) { return c * u * (1.0 - u) * (u - a); }
static double rxn_d(double c, double a, double u) { return c * (-3.0 * u * u + 2.0 * (1.0 + a) * u - a); }

/* R(v) - R(u) for R' = r, with w = v - u factored out of every difference. */
static double rxn_int_diff(double c, double a, double u, double v, double w) {
  double s = v + u, q2 = v * v + u * u, q3 = v * v + v * u + u * u;
  return c * w * (-s * q2 / 4.0 + (1.0 + a) * q3 / 3.0 - a * s / 2.0);
}

void or_step_residual(const or_level* lv, const double* mass, const double* Kst,
                      const double* u, const double* u_prev, double* F) {
  int n = or_nodes(lv);
  double dt = lv->T / lv->m;
  or_stiff_apply(lv, Kst, u, F);
  for (int i = 0; i < n; ++i)
    F[i] += mass[i] / dt * (u[i] - u_prev[i]) - mass[i] * rxn(lv->c, lv->a, u[i]);
}

static void hess_apply(const or_level* lv, const double* mass, const double* Kst,
                       const double* u_lin, const double* v, double* y) {
  int n = or_nodes(lv);
  double dt = lv->T / lv->m;
  or_stiff_apply(lv, Kst, v, y);
  for (int i = 0; i < n; ++i) y[i] += (mass[i] / dt - mass[i] * rxn_d(lv->c, lv->a, u_lin[i])) * v[i];
}

static double dot(int n, const double* a, const double* b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

int or_newton_cg(int n, const double* mass, const double* Kst, const or_level* lv,
                 const double* u_lin, const double* F, double* d, int* truncated) {
  int no = lv->dim == 3 ? 27 : 9, ctr = lv->dim == 3 ? 13 : 4;
  double dt = lv->T / lv->m;
  double* pinv = malloc(sizeof(double) * n);
  double* r = malloc(sizeof(double) * n);
  double* z = malloc(sizeof(double) * n);
  double* p = malloc(sizeof(double) * n);
  double* q = malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) {
    double dg = mass[i] / dt - mass[i] * rxn_d(lv->c, lv->a, u_lin[i]) + Kst[(size_t)i * no + ctr];
    pinv[i] = 1.0 / fabs(dg);
  }
  memset(d, 0, sizeof(double) * n);
  for (int i = 0; i < n; ++i) { r[i] = -F[i]; z[i] = pinv[i] * r[i]; p[i] = z[i]; }
  double rz = dot(n, r, z);
  double r0 = sqrt(rz);
  int it = 0, ret = -1;
  *truncated = 0;
  if (r0 == 0.0) { ret = 0; goto done; }
  for (it = 1; it <= lv->lin_max; ++it) {
    hess_apply(lv, mass, Kst, u_lin, p, q);
    double pq = dot(n, p, q);
    if (pq <= 0.0) {
      *truncated = 1;
      if (it == 1) memcpy(d, z, sizeof(double) * n);
      ret = it;
      break;
    }
    double alpha = rz / pq;
    for (int i = 0; i < n; ++i) { d[i] += alpha * p[i]; r[i] -= alpha * q[i]; z[i] = pinv[i] * r[i]; }
    double rz_new = dot(n, r, z);
    if (sqrt(rz_new) <= lv->lin_rtol * r0) { ret = it; break; }
    double beta = rz_new / rz;
    for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rz = rz_new;
  }
done:
  free(pinv); free(r); free(z); free(p); free(q);
  return ret;
}

/* E(u + alpha d) - E(u), given Ku = K u and Kd = K d. */
static double energy_change(const or_level* lv, int n, const double* mass, const double* u,
                            const double* up, const double* d, const double* Ku,
                            const double* Kd, double alpha) {
  double dt = lv->T / lv->m;
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double w = alpha * d[i];
    double v = u[i] + w;
    s += mass[i] * w * (2.0 * (u[i] - up[i]) + w) / (2.0 * dt);
    s += w * Ku[i] + 0.5 * w * alpha * Kd[i];
    s -= mass[i] * rxn_int_diff(lv->c, lv->a, u[i], v, w);
  }
  return s;
}

int or_step_solve(const or_level* lv, const double* mass, const double* Kst,
                  const double* up, double* u, int* stats) {
  int n = or_nodes(lv);
  double* F = malloc(sizeof(double) * n);
  double* d = malloc(sizeof(double) * n);
  double* Ku = malloc(sizeof(double) * n);
  double* Kd = malloc(sizeof(double) * n);
  int it, conv = 0, cg_total = 0, trunc_total = 0, halvings = 0;
  double dt = lv->T / lv->m;
  double rmax = lv->c * ((1.0 + lv->a) * (1.0 + lv->a) / 3.0 - lv->a);
  double step_max = dt * rmax > 2.0 ? 0.1 : INFINITY;
  memcpy(u, up, sizeof(double) * n);
  for (it = 1; it <= lv->newton_max; ++it) {
    or_step_residual(lv, mass, Kst, u, up, F);
    int tr;
    int cg = or_newton_cg(n, mass, Kst, lv, u, F, d, &tr);
    if (cg < 0) break;
    cg_total += cg; trunc_total += tr;
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) if (fabs(d[i]) > dmax) dmax = fabs(d[i]);
    double alpha = 1.0;
    if (dmax > step_max) {
      /* max-norm trust region: clip every component to [-step_max, step_max];
         if the clipped direction is not a descent direction of E, scale the
         whole direction to max |d| = step_max instead */
      double gdc = 0.0;
      for (int i = 0; i < n; ++i) gdc += F[i] * fmin(fmax(d[i], -step_max), step_max);
      if (gdc < 0.0) {
        for (int i = 0; i < n; ++i) d[i] = fmin(fmax(d[i], -step_max), step_max);
      } else {
        alpha = step_max / dmax;
      }
    }
    if (dmax > lv->newton_tol && dmax > 1e-6) {
      double gd = dot(n, F, d);
      or_stiff_apply(lv, Kst, u, Ku);
      or_stiff_apply(lv, Kst, d, Kd);
      for (int h = 0; h < 40; ++h) {
        double dE = energy_change(lv, n, mass, u, up, d, Ku, Kd, alpha);
        if (dE <= 1e-4 * alpha * gd) break;
        alpha *= 0.5;
        ++halvings;
      }
    }
    for (int i = 0; i < n; ++i) u[i] += alpha * d[i];
    if (dmax <= lv->newton_tol) { conv = 1; break; }
  }
  if (stats) { stats[0] = it; stats[1] = cg_total; stats[2] = trunc_total; stats[3] = halvings; }
  free(F); free(d); free(Ku); free(Kd);
  return conv ? it : -1;
}

void or_activation(int nodes, int m, double dt, double T, const double* slab, double* t_act) {
  for (int i = 0; i < nodes; ++i) {
    double t = T;
    if (slab[i] >= 0.5) {
      t = 0.0;
    } else {
      for (int k = 1; k <= m; ++k) {
        double uk = slab[(size_t)k * nodes + i];
        if (uk >= 0.5) {
          double up = slab[(size_t)(k - 1) * nodes + i];
          t = (double)(k - 1) * dt + dt * (0.5 - up) / (uk - up);
          break;
        }
      }
    }
    t_act[i] = t;
  }
}

int or_solve_sample(const or_level* lv, const double* Z, const double* u0, double* slab,
                    double* t_act, int* newton_per_step) {
  int n = or_nodes(lv), no = lv->dim == 3 ? 27 : 9;
  double* mass = malloc(sizeof(double) * n);
  double* Kst = malloc(sizeof(double) * (size_t)n * no);
  or_assemble(lv, Z, mass, Kst);
  if (u0) memcpy(slab, u0, sizeof(double) * n); else or_initial(lv, slab);
  int total = 0, ret = 0;
  for (int k = 1; k <= lv->m && ret == 0; ++k) {
    int st[4];
    int it = or_step_solve(lv, mass, Kst, slab + (size_t)(k - 1) * n, slab + (size_t)k * n, st);
    if (newton_per_step) newton_per_step[k - 1] = st[0];
    total += st[0];
    if (it < 0) ret = -k;
  }
  if (t_act) or_activation(n, lv->m, lv->T / lv->m, lv->T, slab, t_act);
  free(mass); free(Kst);
  return ret ? ret : total;
}

void or_slab_residual(const or_level* lv, const double* mass, const double* Kst,
                      const double* slab, double* F) {
  int n = or_nodes(lv);
  for (int k = 1; k <= lv->m; ++k)
    or_step_residual(lv, mass, Kst, slab + (size_t)k * n, slab + (size_t)(k - 1) * n,
                     F + (size_t)(k - 1) * n);
}
