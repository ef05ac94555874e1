/*
 * Oracle: the nonlinear space-time problem of one sample (Sec. 3.3,
 * Eq. mono_disc) in the implicit-Euler variant, solved step by step.
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * Block row k of the space-time system (k = 1..m, dt = T/m, M lumped), divided
 * by dt:
 *   F_k(u) = (M/dt)(u_k - u_{k-1}) + K (theta u_k + (1-theta) u_{k-1})
 *            - M r(u_k) - M s_k,                 r(u) = c u (1-u)(u-a)
 * (the FHN current of Eq. ionic_term written as -c u(1-u)(u-a) on [0,1]);
 * theta = 1 is implicit Euler, theta = 1/2 the Crank-Nicolson blocks of
 * Sec. 3.2 (Eq. st-system: A = M + dt/2 K, B = -M + dt/2 K) with the reaction
 * of Sec. 3.3 (Eq. mono_disc, r(u) = dt (I x M) I_ion(u)) at the new time
 * level; s_k is the applied current averaged over the step.
 * Its Jacobian block (Sec. 3.3) is  H = M/dt + theta K - M diag(r'(u)),
 *   r'(u) = c(-3u^2 + 2(1+a)u - a).
 * H is symmetric, so F_k is the gradient of the step energy
 *   E(u) = (u-u_{k-1})^T M (u-u_{k-1}) / (2dt) + theta u^T K u / 2
 *          + (1-theta) u_{k-1}^T K u - sum_i m_i (R(u_i) + s_k,i u_i),   R' = r,
 * and H is its Hessian.  When c dt max r' > 1 (max r' = c((1+a)^2/3 - a)) the
 * step has several roots -- local minima of E -- and the paper is silent on
 * which one the scheme means.  The root is defined as the end point of the
 * gradient flow of E in the mass metric started at u_{k-1},
 *   M v' = -F_k(v),  v(0) = u_{k-1},
 * the minimum in whose basin of attraction u_{k-1} lies: a definition with no
 * solver in it.  or_step_gradient_flow computes it plainly (fixed, strictly
 * convex implicit-Euler pseudo-steps); or_step_solve reaches the same point
 * faster by a gradient-flow continuation, and the tests pin the two together:
 *   - linearly implicit pseudo-steps (M/t + H(u)) d = -F(u), u += d, by
 *     Jacobi-preconditioned CG; t starts at 1/(2 max r'); a step whose CG
 *     meets non-positive curvature (M/t + H not positive definite) is retried
 *     with t/4.  A step with M/t + H
 *     positive definite never reverses the sign of the flow's unstable
 *     component near a saddle (the linearised step multiplies it by
 *     1/(1 - t lambda_u) > 0), so it does not jump between basins, and t can
 *     grow as far as the local curvature allows -- near a nearly degenerate
 *     saddle, where the flow crawls, that is what makes the continuation fast;
 *   - a step that would move some node by more than FLOW_MOVE is taken
 *     shortened to that move and the next t is scaled down accordingly
 *     (counted as a halving); otherwise t grows towards the move limit, at
 *     most doubling;
 *   - once an accepted step moves no node by more than FLOW_NEWTON the flow has
 *     arrived near its minimum, and Newton steps (t = infinity) finish it as
 *     long as their CG meets no non-positive curvature and they move no node
 *     by more than 10 FLOW_NEWTON; otherwise the flow resumes;
 *   - stop when an accepted step moves no node by more than newton_tol.
 * Where c dt max r' <= 1, H is positive definite for every state, the root is
 * unique, and plain Newton-CG with Armijo backtracking on E (sigma = 1e-4,
 * halving, at most 40; full step when max|d| <= 1e-6) computes it.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* Parameters of the gradient-flow continuation (see or_step_solve). */
#define FLOW_MOVE 0.3     /* largest nodal move of an accepted pseudo-step          */
#define FLOW_TMIN 1e-9    /* pseudo-steps this short are accepted regardless        */
#define FLOW_TMAX 1e20    /* upper bound of the growing pseudo-step                 */
#define FLOW_NEWTON 1e-2  /* accepted move below which Newton steps finish the step  */

static double rxn(double c, double a, double u) { return c * u * (1.0 - u) * (u - a); }
static double rxn_d(double c, double a, double u) { return c * (-3.0 * u * u + 2.0 * (1.0 + a) * u - a); }

/* R(v) - R(u) for R' = r, with w = v - u factored out of every difference. */
static double rxn_int_diff(double c, double a, double u, double v, double w) {
  double s = v + u, q2 = v * v + u * u, q3 = v * v + v * u + u * u;
  return c * w * (-s * q2 / 4.0 + (1.0 + a) * q3 / 3.0 - a * s / 2.0);
}

static double theta_of(const or_level* lv) { return lv->scheme == 1 ? 0.5 : 1.0; }

void or_step_residual(const or_level* lv, const double* mass, const double* Kst,
                      const double* u, const double* u_prev, int k, double* F) {
  int n = or_nodes(lv);
  double dt = lv->T / lv->m, th = theta_of(lv);
  double* Kp = malloc(sizeof(double) * n);
  double* sk = malloc(sizeof(double) * n);
  or_stiff_apply(lv, Kst, u, F);
  or_stiff_apply(lv, Kst, u_prev, Kp);
  or_stimulus_step(lv, k, sk);
  for (int i = 0; i < n; ++i)
    F[i] = th * F[i] + (1.0 - th) * Kp[i] + mass[i] / dt * (u[i] - u_prev[i]) -
           mass[i] * rxn(lv->c, lv->a, u[i]) - mass[i] * sk[i];
  free(Kp); free(sk);
}

/* y = H v, H = M/dt + theta K - M diag(r'(u_lin)) */
static void hess_apply(const or_level* lv, const double* mass, const double* Kst,
                       const double* u_lin, const double* v, double* y) {
  int n = or_nodes(lv);
  double dt = lv->T / lv->m, th = theta_of(lv);
  or_stiff_apply(lv, Kst, v, y);
  for (int i = 0; i < n; ++i)
    y[i] = th * y[i] + (mass[i] / dt - mass[i] * rxn_d(lv->c, lv->a, u_lin[i])) * v[i];
}

static double dot(int n, const double* a, const double* b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Jacobi-preconditioned CG on (H + shift M) d = -F from d = 0, H the step
 * Hessian at u_lin; truncated at the first search direction with p^T A p <= 0
 * (then the current iterate, or the preconditioned steepest-descent step if
 * that happens in the first iteration).  shift = 0: the Newton system. */
static int shifted_cg(int n, const double* mass, const double* Kst, const or_level* lv,
                      const double* u_lin, double shift, const double* F, double* d,
                      int* truncated) {
  int no = or_n_offsets(lv->dim), ctr = (no - 1) / 2;
  double dt = lv->T / lv->m;
  double* pinv = malloc(sizeof(double) * n);
  double* r = malloc(sizeof(double) * n);
  double* z = malloc(sizeof(double) * n);
  double* p = malloc(sizeof(double) * n);
  double* q = malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) {
    double dg = mass[i] * (shift + 1.0 / dt) - mass[i] * rxn_d(lv->c, lv->a, u_lin[i]) +
                theta_of(lv) * Kst[(size_t)i * no + ctr];
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
    for (int i = 0; i < n; ++i) q[i] += shift * mass[i] * p[i];
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

int or_newton_cg(int n, const double* mass, const double* Kst, const or_level* lv,
                 const double* u_lin, const double* F, double* d, int* truncated) {
  return shifted_cg(n, mass, Kst, lv, u_lin, 0.0, F, d, truncated);
}

/* E(u + alpha d) - E(u) for the step energy
 *   E(u) = (u-up)^T M (u-up)/(2dt) + theta u^T K u/2 + (1-theta) up^T K u
 *          - sum_i m_i (R(u_i) + s_i u_i),
 * given Ku = K u, Kd = K d, Kp = K up and the step's applied current s. */
static double energy_change(const or_level* lv, int n, const double* mass, const double* u,
                            const double* up, const double* d, const double* Ku,
                            const double* Kd, const double* Kp, const double* sk, double alpha) {
  double dt = lv->T / lv->m, th = theta_of(lv);
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double w = alpha * d[i];
    double v = u[i] + w;
    s += mass[i] * w * (2.0 * (u[i] - up[i]) + w) / (2.0 * dt);
    s += th * (w * Ku[i] + 0.5 * w * alpha * Kd[i]) + (1.0 - th) * w * Kp[i];
    s -= mass[i] * rxn_int_diff(lv->c, lv->a, u[i], v, w) + mass[i] * sk[i] * w;
  }
  return s;
}

int or_step_solve(const or_level* lv, const double* mass, const double* Kst,
                  const double* up, int k, double* u, int* stats) {
  int n = or_nodes(lv);
  double* F = malloc(sizeof(double) * n);
  double* d = malloc(sizeof(double) * n);
  double* Ku = malloc(sizeof(double) * n);
  double* Kd = malloc(sizeof(double) * n);
  double* Kp = malloc(sizeof(double) * n);
  double* sk = malloc(sizeof(double) * n);
  or_stiff_apply(lv, Kst, up, Kp);
  or_stimulus_step(lv, k, sk);
  int it, conv = 0, cg_total = 0, trunc_total = 0, halvings = 0;
  double dt = lv->T / lv->m;
  double rmax = lv->c * ((1.0 + lv->a) * (1.0 + lv->a) / 3.0 - lv->a);
  const int flow = dt * rmax > 1.0;
  double tau = 0.5 / rmax, sw = FLOW_NEWTON;
  int newton_phase = 0;
  memcpy(u, up, sizeof(double) * n);
  for (it = 1; it <= lv->newton_max; ++it) {
    or_step_residual(lv, mass, Kst, u, up, k, F);
    int tr;
    if (flow) {
      /* linearly implicit pseudo-step of the gradient flow M v' = -F(v):
         (M/t + H(u)) d = -F(u), kept only if its CG met positive curvature
         throughout (M/t + H positive definite); once the flow has (nearly)
         arrived (an accepted move below FLOW_NEWTON), Newton steps
         (t = infinity) finish the solve as long as their CG meets no
         non-positive curvature and they move no node by more than
         10 FLOW_NEWTON; a Newton step that fails either test is discarded and
         the flow resumes with a tighter switch threshold */
      const double t = tau;
      int cg = shifted_cg(n, mass, Kst, lv, u, newton_phase ? 0.0 : 1.0 / t, F, d, &tr);
      if (cg < 0) break;
      cg_total += cg; trunc_total += tr;
      double dmax = 0.0;
      for (int i = 0; i < n; ++i) if (fabs(d[i]) > dmax) dmax = fabs(d[i]);
      if (!newton_phase && tr && t > FLOW_TMIN) {
        /* M/t + H is not positive definite: retry with a quarter of t */
        tau = 0.25 * t;
        ++halvings;
        continue;
      }
      if (newton_phase) {
        if (tr || dmax > 10.0 * sw) {
          newton_phase = 0;
          sw *= 0.1;
          ++halvings;
          continue;
        }
        for (int i = 0; i < n; ++i) u[i] += d[i];
        if (dmax <= lv->newton_tol) { conv = 1; break; }
        continue;
      }
      if (dmax > FLOW_MOVE && t > FLOW_TMIN) {
        /* the step would move a node by more than FLOW_MOVE: take it shortened
           to that move (a positive multiple of the step keeps its sign along
           every eigenvector of M/t + H) and continue with a shorter pseudo-step */
        const double sc = FLOW_MOVE / dmax;
        for (int i = 0; i < n; ++i) u[i] += sc * d[i];
        tau = t * 0.9 * sc;
        ++halvings;
        continue;
      }
      for (int i = 0; i < n; ++i) u[i] += d[i];
      if (dmax <= lv->newton_tol) { conv = 1; break; }
      if (dmax <= sw) newton_phase = 1;
      /* grow towards the move limit, at most doubling */
      tau = fmin(t * fmin(2.0, 0.9 * FLOW_MOVE / dmax), FLOW_TMAX);
      continue;
    }
    int cg = or_newton_cg(n, mass, Kst, lv, u, F, d, &tr);
    if (cg < 0) break;
    cg_total += cg; trunc_total += tr;
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) if (fabs(d[i]) > dmax) dmax = fabs(d[i]);
    double alpha = 1.0;
    if (dmax > lv->newton_tol && dmax > 1e-6) {
      double gd = dot(n, F, d);
      or_stiff_apply(lv, Kst, u, Ku);
      or_stiff_apply(lv, Kst, d, Kd);
      for (int h = 0; h < 40; ++h) {
        double dE = energy_change(lv, n, mass, u, up, d, Ku, Kd, Kp, sk, alpha);
        if (dE <= 1e-4 * alpha * gd) break;
        alpha *= 0.5;
        ++halvings;
      }
    }
    for (int i = 0; i < n; ++i) u[i] += alpha * d[i];
    if (dmax <= lv->newton_tol) { conv = 1; break; }
  }
  if (stats) { stats[0] = it; stats[1] = cg_total; stats[2] = trunc_total; stats[3] = halvings; }
  free(F); free(d); free(Ku); free(Kd); free(Kp); free(sk);
  return conv ? it : -1;
}

/*
 * A solver-independent definition of the root of one step: the end point of
 * the gradient flow of the step energy E (in the mass metric) started at
 * u_{k-1},
 *     M v'(s) = -F_k(v(s)),   v(0) = u_{k-1}  (or a given v0),
 * i.e. the local minimum of E in whose basin of attraction u_{k-1} lies.  The
 * flow is integrated by implicit-Euler pseudo-steps of fixed length tau,
 *     v_{j+1} = argmin_w  E(w) + (w - v_j)^T M (w - v_j) / (2 tau),
 * each of them a strictly convex problem when tau (max r' - 1/dt) < 1 (its
 * Hessian M/tau + M/dt + K - M diag(r'(w)) is then positive definite, K being
 * positive semidefinite), so every pseudo-step has exactly one solution, found
 * by Newton's method with a CG solve to 1e-14 and backtracking on the convex
 * objective.  No truncation, clipping, preconditioner or step-size choice
 * enters the result.  Once max_i |F_k(v)_i| / m_i <= 1e-8 the flow is within
 * ~1e-9 of a nondegenerate minimum -- far inside Newton's region of quadratic
 * convergence around it -- and plain Newton steps (the Hessian there is
 * positive definite; a CG that meets non-positive curvature is a failure)
 * finish the solve until max_i |F_k(v)_i| / m_i <= ftol.
 * stats = {pseudo-steps, Newton iterations, CG iterations}.  Returns the
 * pseudo-steps taken, or -1.
 */
static int prox_cg(int n, const double* mass, const double* Kst, const or_level* lv,
                   const double* w, double inv_tau, const double* G, double* d) {
  int no = or_n_offsets(lv->dim), ctr = (no - 1) / 2;
  double dt = lv->T / lv->m;
  double* pinv = malloc(sizeof(double) * n);
  double* r = malloc(sizeof(double) * n);
  double* z = malloc(sizeof(double) * n);
  double* p = malloc(sizeof(double) * n);
  double* q = malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i)
    pinv[i] = 1.0 / (mass[i] * (inv_tau + 1.0 / dt - rxn_d(lv->c, lv->a, w[i])) +
                     theta_of(lv) * Kst[(size_t)i * no + ctr]);
  memset(d, 0, sizeof(double) * n);
  for (int i = 0; i < n; ++i) { r[i] = -G[i]; z[i] = pinv[i] * r[i]; p[i] = z[i]; }
  double rz = dot(n, r, z), r0 = sqrt(rz);
  int it = 0, ret = -1;
  if (r0 == 0.0) { ret = 0; goto done; }
  for (it = 1; it <= 20 * n + 100; ++it) {
    hess_apply(lv, mass, Kst, w, p, q);
    for (int i = 0; i < n; ++i) q[i] += mass[i] * inv_tau * p[i];
    double pq = dot(n, p, q);
    if (!(pq > 0.0)) break;   /* cannot happen for a positive definite Hessian */
    double alpha = rz / pq;
    for (int i = 0; i < n; ++i) { d[i] += alpha * p[i]; r[i] -= alpha * q[i]; z[i] = pinv[i] * r[i]; }
    double rz_new = dot(n, r, z);
    if (sqrt(rz_new) <= 1e-14 * r0) { ret = it; break; }
    double beta = rz_new / rz;
    for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rz = rz_new;
  }
done:
  free(pinv); free(r); free(z); free(p); free(q);
  return ret;
}

int or_step_gradient_flow(const or_level* lv, const double* mass, const double* Kst,
                          const double* up, int k, const double* v0, double* u, double tau,
                          double ftol, int max_pseudo, int* stats) {
  int n = or_nodes(lv);
  double dt = lv->T / lv->m;
  double rmax = lv->c * ((1.0 + lv->a) * (1.0 + lv->a) / 3.0 - lv->a);
  if (!(tau > 0.0) || tau * (rmax - 1.0 / dt) >= 1.0) return -1;   /* not strictly convex */
  double* v = malloc(sizeof(double) * n);
  double* F = malloc(sizeof(double) * n);
  double* G = malloc(sizeof(double) * n);
  double* d = malloc(sizeof(double) * n);
  double* Ku = malloc(sizeof(double) * n);
  double* Kd = malloc(sizeof(double) * n);
  double* Kp = malloc(sizeof(double) * n);
  double* sk = malloc(sizeof(double) * n);
  or_stiff_apply(lv, Kst, up, Kp);
  or_stimulus_step(lv, k, sk);
  int j, ok = 0, newton = 0, cg = 0;
  double inv_tau = 1.0 / tau;
  memcpy(u, v0 ? v0 : up, sizeof(double) * n);
  const double flow_tol = ftol > 1e-8 ? ftol : 1e-8;
  for (j = 0; j <= max_pseudo; ++j) {
    or_step_residual(lv, mass, Kst, u, up, k, F);
    double fm = 0.0;
    for (int i = 0; i < n; ++i) if (fabs(F[i]) / mass[i] > fm) fm = fabs(F[i]) / mass[i];
    if (fm <= flow_tol) { ok = 1; break; }
    if (j == max_pseudo) break;
    memcpy(v, u, sizeof(double) * n);
    /* Newton on the strictly convex pseudo-step objective
       P(w) = E(w) + (w - v)^T M (w - v) / (2 tau),  gradient F(w) + M (w - v) / tau */
    int conv = 0;
    for (int it = 0; it < 100 && !conv; ++it) {
      if (it > 0) or_step_residual(lv, mass, Kst, u, up, k, F);
      for (int i = 0; i < n; ++i) G[i] = F[i] + mass[i] * inv_tau * (u[i] - v[i]);
      int c1 = prox_cg(n, mass, Kst, lv, u, inv_tau, G, d);
      if (c1 < 0) goto fail;
      cg += c1;
      ++newton;
      double dmax = 0.0;
      for (int i = 0; i < n; ++i) if (fabs(d[i]) > dmax) dmax = fabs(d[i]);
      double alpha = 1.0;
      if (dmax > 1e-8) {
        double gd = dot(n, G, d);
        or_stiff_apply(lv, Kst, u, Ku);
        or_stiff_apply(lv, Kst, d, Kd);
        for (int h = 0; h < 60; ++h) {
          double dP = energy_change(lv, n, mass, u, up, d, Ku, Kd, Kp, sk, alpha);
          for (int i = 0; i < n; ++i) {
            double w = alpha * d[i];
            dP += mass[i] * w * (2.0 * (u[i] - v[i]) + w) * 0.5 * inv_tau;
          }
          if (dP <= 1e-4 * alpha * gd) break;
          alpha *= 0.5;
        }
      }
      for (int i = 0; i < n; ++i) u[i] += alpha * d[i];
      if (dmax <= 1e-13) conv = 1;
    }
    if (!conv) goto fail;
  }
  if (ok && flow_tol > ftol) {
    /* Newton polish at the nondegenerate minimum the flow has reached */
    ok = 0;
    for (int it = 0; it < 50; ++it) {
      or_step_residual(lv, mass, Kst, u, up, k, F);
      double fm = 0.0;
      for (int i = 0; i < n; ++i) if (fabs(F[i]) / mass[i] > fm) fm = fabs(F[i]) / mass[i];
      if (fm <= ftol) { ok = 1; break; }
      int c1 = prox_cg(n, mass, Kst, lv, u, 0.0, F, d);
      if (c1 < 0) break;
      cg += c1;
      ++newton;
      for (int i = 0; i < n; ++i) u[i] += d[i];
    }
  }
fail:
  if (stats) { stats[0] = j; stats[1] = newton; stats[2] = cg; }
  free(v); free(F); free(G); free(d); free(Ku); free(Kd); free(Kp); free(sk);
  return ok ? j : -1;
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
  int n = or_nodes(lv), no = or_n_offsets(lv->dim);
  double* mass = malloc(sizeof(double) * n);
  double* Kst = malloc(sizeof(double) * (size_t)n * no);
  or_assemble(lv, Z, mass, Kst);
  if (u0) memcpy(slab, u0, sizeof(double) * n); else or_initial(lv, slab);
  int total = 0, ret = 0;
  for (int k = 1; k <= lv->m && ret == 0; ++k) {
    int st[4];
    int it = or_step_solve(lv, mass, Kst, slab + (size_t)(k - 1) * n, k, slab + (size_t)k * n, st);
    if (newton_per_step) newton_per_step[k - 1] = st[0];
    total += st[0];
    if (it < 0) ret = -k;
  }
  if (t_act) {
    if (lv->qoi == 1) memcpy(t_act, slab + (size_t)lv->m * n, sizeof(double) * n);
    else or_activation(n, lv->m, lv->T / lv->m, lv->T, slab, t_act);
  }
  free(mass); free(Kst);
  return ret ? ret : total;
}

void or_slab_residual(const or_level* lv, const double* mass, const double* Kst,
                      const double* slab, double* F) {
  int n = or_nodes(lv);
  for (int k = 1; k <= lv->m; ++k)
    or_step_residual(lv, mass, Kst, slab + (size_t)k * n, slab + (size_t)(k - 1) * n, k,
                     F + (size_t)(k - 1) * n);
}
