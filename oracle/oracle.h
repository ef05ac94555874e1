/*
 * Oracle for the space-time MLMC monodomain path: plain, slow, FP64 CPU code.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes, links or
 * calls this code; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA implementation.
 *
 * Every function follows a passage of arXiv:1911.06066 ("Space-time multilevel
 * Monte Carlo methods and their application to cardiac electrophysiology"),
 * cited by section / equation, in the variant the workloads fix:
 * Q1 elements with lumped mass, implicit Euler, lognormal KL conductivity with a
 * separable exponential covariance, anisotropic fiber tensor, activation time.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

/* ---------- counter-based generator (Salmon et al., SC'11) ---------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_log(double x);                       /* own ln, atanh series          */
void or_sincos_2pi(double u, double* s, double* c); /* sin/cos of 2*pi*u      */
/* xi[0..M) for (seed, level pair, sample id): standard normals, Box-Muller.   */
void or_xi(uint64_t seed, int level, uint64_t sample_id, int M, double* xi);

/* psi[0..M) ~ U(-1, 1) for (seed, level pair, sample id), the same counters. */
void or_psi_uniform(uint64_t seed, int level, uint64_t sample_id, int M, double* psi);

/* ---------- Karhunen-Loeve expansion (Sec. 3.1.1, Eq. KL-expansion) ---------- */
/* 1D eigenpairs of exp(-|x-y|/ell) on an interval of length len, modes 0..n-1
 * (decreasing eigenvalue).  omega[n], lam[n] (unit variance), nrm[n] = the
 * normalisation divisor; odd modes are sine modes. */
void or_kl_1d(double len, double ell, int n, double* omega, double* lam, double* nrm);
/* Value of 1D mode k at x in [0, len]. */
double or_kl_phi_1d(double len, int k, double omega, double nrm, double x);
/* Multi-D mode table: the M largest products sigma2*prod(lam_i), ties broken by
 * index sum then lexicographic.  idx[3*k..] = 1D indices, sqrt_lam[k]. */
int or_kl_table(int dim, const double* L, double sigma2, double ell, int M,
                int* idx, double* sqrt_lam);
/* Z on cell centroids of an (nx,ny,nz) grid for nsamp samples.
 * xi: [nsamp][M]; Z: [nsamp][cells]. */
int or_kl_field(int dim, const double* L, const int* n, double sigma2, double ell,
                int M, int nsamp, const double* xi, double* Z);

/* The paper's KL variant (kl_affine.c): pivoted Cholesky of the Gaussian
 * covariance sigma2 exp(-|x-x'|^2/ell^2) on n candidate points X[n][dim], at
 * most M columns, stopped at a remainder trace <= tol times the full trace.
 * piv[M] pivot indices, Lpiv[M][M] the pivot rows of the factor (lower
 * triangular), L[n][M] (may be NULL) the factor.  Returns the rank m. */
int or_pivoted_cholesky(int dim, int n, const double* X, double sigma2, double ell, int M,
                        double tol, int* piv, double* Lpiv, double* L);
/* The factor's columns at any points Y[ny][dim] (Nystrom extension from the
 * pivot points Xp[m][dim] and Lpiv): Phi[ny][M] (columns >= m zero). */
void or_pc_eval(int dim, int ny, const double* Y, const double* Xp, double sigma2, double ell,
                int M, int m, const double* Lpiv, double* Phi);

/* ---------- one discretisation level --------------------------------------- */
typedef struct {
  int dim;            /* 1, 2 or 3                                             */
  int n[3];           /* cells per axis (n[2] ignored in 2D)                    */
  int m;              /* implicit-Euler steps                                   */
  double L[3];        /* domain extents                                         */
  double T;           /* end time                                               */
  double c, a;        /* reaction c*u(1-u)(u-a)                                 */
  double s_t, s_l0;   /* D = s_t I + (s_l - s_t) f f^T,  s_l = s_l0 exp(Z)      */
  double theta0, theta1; /* fiber angle in degrees; 3D: linear in z             */
  double stim_r;      /* u0 = 1 inside |x - x_c| < stim_r                       */
  double stim_c[3];
  double newton_tol;  /* stop when max|delta| <= newton_tol                     */
  int newton_max;
  double lin_rtol;    /* CG relative tolerance (preconditioned residual)        */
  int lin_max;
  int scheme;         /* 0: implicit Euler; 1: Crank-Nicolson diffusion with the
                         reaction at the new time level (Sec. 3.2-3.3)           */
  int stim_kind;      /* 0: u0 = 1 in the ball; 1: u0 = 0 and the applied current
                         I_app = stim_amp exp(-|x - stim_c|^2 / stim_sigma^2)
                         for 0 <= t < stim_t1 (Sec. 4 set-up)                    */
  double stim_amp, stim_sigma, stim_t1;
  int qoi;            /* 0: activation time; 1: the final state u(T)            */
  int cond_kind;      /* 0: D = s_t I + (s_l0 e^Z - s_t) f f^T (fiber, lognormal);
                         1: D = s_l0 (1 + Z) I (the paper's affine isotropic G)  */
} or_level;

int or_nodes(const or_level* lv);
int or_cells(const or_level* lv);
int or_n_offsets(int dim);   /* 3^dim */
/* Lumped mass (row sums of the Q1 consistent mass), stiffness stored per node
 * as 3^dim couplings to offsets in {-1,0,1}^dim (x fastest). */
void or_assemble(const or_level* lv, const double* Z, double* mass, double* Kst);
void or_stiff_apply(const or_level* lv, const double* Kst, const double* v, double* y);
void or_initial(const or_level* lv, double* u0);
/* Per-step residual F(u; u_prev) of step k (1-based; the applied current
 * enters through its average over [t_{k-1}, t_k]):
 *   F = (M/dt)(u - u_prev) + K (theta u + (1-theta) u_prev) - M r(u) - M s_k,
 * theta = 1 (implicit Euler) or 1/2 (Crank-Nicolson). */
void or_step_residual(const or_level* lv, const double* mass, const double* Kst,
                      const double* u, const double* u_prev, int k, double* F);
/* The applied current's average over step k at every node (0 for stim_kind 0). */
void or_stimulus_step(const or_level* lv, int k, double* s);
/* Newton direction: Jacobi-PCG on H d = -F, truncated on negative curvature.
 * Returns CG iterations (<0: lin_max reached); *truncated set if truncated. */
int or_newton_cg(int n, const double* mass, const double* Kst, const or_level* lv,
                 const double* u_lin, const double* F, double* d, int* truncated);
/* One implicit-Euler step from up by line-search Newton-CG on the step energy.
 * stats = {newton its, cg its, truncations, halvings}.  Returns its or -1. */
int or_step_solve(const or_level* lv, const double* mass, const double* Kst,
                  const double* up, int k, double* u, int* stats);
/* Solver-independent root of one step: the end point of the mass-metric
 * gradient flow M v' = -F(v) of the step energy from v(0) = up (or v0 when not
 * NULL), integrated by
 * strictly convex implicit-Euler pseudo-steps of length tau (requires
 * tau (max r' - 1/dt) < 1) until max|F_i| / m_i <= ftol.  stats = {pseudo-steps,
 * Newton iterations, CG iterations}.  Returns pseudo-steps, or -1. */
int or_step_gradient_flow(const or_level* lv, const double* mass, const double* Kst,
                          const double* up, int k, const double* v0, double* u, double tau,
                          double ftol, int max_pseudo, int* stats);
/* Sequential time stepping for one sample.  u0 = NULL: the configured initial
 * state (the stimulus ball, or 0 with the applied current).
 * slab: [m+1][nodes] (slice 0 = u0), t_act: [nodes] = the quantity of
 * interest (activation times, or u(T) when lv->qoi == 1).
 * Returns total Newton iterations, or -(k) if step k failed to converge. */
int or_solve_sample(const or_level* lv, const double* Z, const double* u0, double* slab,
                    double* t_act, int* newton_per_step);
/* All-at-once space-time residual of the slab (Eq. mono_disc; implicit-Euler
 * or Crank-Nicolson blocks). */
void or_slab_residual(const or_level* lv, const double* mass, const double* Kst,
                      const double* slab, double* F);
/* Activation time: first crossing of 0.5, linear in time; T if none. */
void or_activation(int nodes, int m, double dt, double T, const double* slab,
                   double* t_act);

/* ---------- MLMC (Sec. 3.1.2, Eqs. MC-estimator, MLMC-estimator) -------------- */
/* Injection of a level-l nodal field onto the coarsest grid (level 0). */
void or_inject(const or_level* fine, const or_level* l0, const double* f, double* out);
typedef struct { long n; double* mean; double* m2; } or_welford;
void or_welford_add(or_welford* w, int len, const double* y);
/* One level pair: y = inj(t_l) - inj(t_{l-1}), y2 = inj(t_l)^2 - inj(t_{l-1})^2
 * on the coarsest grid (coarse == NULL on level 0). */
int or_sample_pair(const or_level* fine, const or_level* coarse, const or_level* l0,
                   double sigma2, double ell, int M, uint64_t seed, int level,
                   uint64_t sample_id, double* y, double* y2, int* newton_iters);
#endif
