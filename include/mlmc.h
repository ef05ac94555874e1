/*
 * mlmc.h -- C ABI of the GB300 space-time multilevel Monte Carlo library for
 * the stochastic monodomain equation (arXiv:1911.06066).
 *
 * Problem (Sec. 2.1, Eq. monodomain and Eq. ionic_term; Sec. 3.1.1,
 * Eq. KL-expansion), in the variant this library implements:
 *     u_t = div(D grad u) + c u (1-u) (u-a)   on a box, Neumann boundary,
 *     D   = s_t I + (s_l - s_t) f f^T,  s_l = s_l0 exp(Z),  f = (cos th, sin th, 0),
 *     Z   = sum_k sqrt(lam_k) phi_k(x) xi_k,  xi_k ~ N(0,1) (Philox4x32-10),
 *     u(x,0) = 1 inside the ball |x - x_c| < stim_r, else 0,
 * discretised by Q1 elements with lumped mass and implicit Euler (the block
 * lower-bidiagonal space-time system of Sec. 3.2, Eq. system_C, with the
 * reaction of Sec. 3.3, Eq. mono_disc), solved step by step.  Where a step
 * has several roots (c dt max r' > 1, max r' = c((1+a)^2/3 - a)) the root is
 * the end point of the gradient flow M v' = -F_k(v) of the step's energy
 * started at u_{k-1} -- the local minimum in whose basin u_{k-1} lies -- which
 * the solver reaches by a gradient-flow continuation (linearly implicit
 * pseudo-steps, then Newton); elsewhere the root is unique and Newton with a
 * line search finds it.  The quantity of
 * interest is the activation time (first t with u >= 1/2, linear in t).  Its
 * mean and variance are estimated by MC / MLMC (Sec. 3.1.2, Eq. MC-estimator,
 * Eq. MLMC-estimator).
 *
 * Conventions for every call:
 *   - "device" pointers are CUDA device memory of the current device, owned by
 *     the caller; "host" pointers are host memory owned by the caller.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream);
 *     calls are asynchronous on it unless stated otherwise.
 *   - every call returns an mlmc_status; on error nothing is enqueued and
 *     mlmc_last_error(ctx) describes the failure.  No call aborts the process.
 *   - a context is not thread-safe; use one per host thread.
 *   - node arrays are ordered x fastest, then y, then z; cell arrays likewise.
 *     Level l has n0[d] * 2^l cells per axis and m0 * 2^l time steps.
 */
#ifndef MLMC_H
#define MLMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLMC_MAX_LEVELS 8

typedef enum {
  MLMC_OK = 0,
  MLMC_ERR_ARG = -1,          /* invalid argument or configuration            */
  MLMC_ERR_OOM = -2,          /* device allocation failed                      */
  MLMC_ERR_NOT_CONVERGED = -3,/* a sample's Newton iteration did not converge  */
  MLMC_ERR_TIMEOUT = -4,      /* a bounded device wait ran out                 */
  MLMC_ERR_CUDA = -5,         /* a CUDA runtime call failed                    */
  MLMC_ERR_WORKSPACE = -6,    /* workspace missing, too small or misaligned    */
  MLMC_WARN_BIAS = 1          /* mlmc_run_to_rmse: outputs valid and the sampling
                                 error at its target, but the bias estimate exceeds
                                 eps/sqrt(2), so the RMSE target is not reached    */
} mlmc_status;

typedef enum {
  MLMC_PREC_FP64 = 0,   /* every step in FP64                                       */
  MLMC_PREC_MIXED = 1   /* FP32 Krylov inner solves on levels with c dt max r' <=
                           mixed_cdr_max (FP64 on the others); FP64 residual,
                           update, QoI                                         */
} mlmc_precision;

/* Problem and solver configuration (plain data, copied by mlmc_create). */
typedef struct {
  int dim;               /* 2 or 3                                                  */
  int n_levels;          /* 1 .. MLMC_MAX_LEVELS                                     */
  int n0[3];             /* level-0 cells per axis (n0[2] ignored in 2D)             */
  int m0;                /* level-0 implicit-Euler steps                            */
  double L[3];           /* box extents                                              */
  double T;              /* end time                                                 */
  double c, a;           /* reaction c u (1-u)(u-a)                                  */
  double s_t, s_l0;      /* transverse / longitudinal conductivity                   */
  double theta0_deg;     /* fiber angle; in 3D it varies linearly in z from          */
  double theta1_deg;     /*   theta0 at z = 0 to theta1 at z = L[2]                  */
  double stim_r;         /* stimulus radius and centre                               */
  double stim_c[3];
  double kl_sigma2;      /* KL variance, correlation length, number of modes         */
  double kl_ell;
  int kl_modes;
  int precision;         /* mlmc_precision                                           */
  double newton_tol;     /* stop when an accepted correction moves no node by more
                            than newton_tol                                          */
  int newton_max;        /* nonlinear iterations (Newton or pseudo-steps, accepted or
                            retried) per time step                                  */
  double lin_rtol;       /* CG relative tolerance (FP64 inner solves)                */
  int lin_max;           /* CG iterations per Newton step                            */
  int solver;            /* mlmc_solver: kernel layout of the per-sample sweep        */
  double mixed_cdr_max;  /* MLMC_PREC_MIXED uses FP32 inner solves only on levels with
                            c dt max r' <= mixed_cdr_max (<= 0 selects the default 2);
                            the KL field is synthesised on the tensor cores on those
                            of them with c dt max r' <= 2 */
  int cluster_size;      /* cluster layout: CTAs per sample (1, 2, 4, 8 or 16); 0 picks
                            the smallest that fits shared memory                        */
  int precond;           /* mlmc_precond: preconditioner of the CG inner solves          */
  int mg_nu;             /* MLMC_PRECOND_GMG: smoothing sweeps before and after the coarse
                            correction, 0..8 (0 selects the default 2)                   */
  int mg_coarse_sweeps;  /* MLMC_PRECOND_GMG: smoothing sweeps on the coarsest grid, 0..64
                            (0 selects the default 8)                                    */
  int use_graph;         /* nonzero: mlmc_run / mlmc_run_more / mlmc_run_to_rmse capture
                            their whole multi-stream schedule of one call (every batch of
                            every level) into a CUDA graph and launch it as one unit; the
                            instantiated graph is kept and updated in place when the next
                            call has the same shape.  Ignored on the legacy default stream
                            (stream NULL), which cannot be captured.  Results are
                            identical to the direct launches.                            */
  /* The paper's own time discretisation and stimulus (Sec. 3.2, Eq. st-system;
     Sec. 3.3, Eq. mono_disc; Sec. 4 set-up).  All zero selects the variant
     above (implicit Euler, the ball as initial state, activation times). */
  int time_scheme;       /* mlmc_scheme                                                  */
  int stim_kind;         /* mlmc_stimulus                                                */
  double stim_amp;       /* MLMC_STIM_PULSE: I_app = stim_amp exp(-|x - stim_c|^2 /      */
  double stim_sigma;     /*   stim_sigma^2) for 0 <= t < stim_t1, u(x, 0) = 0; each step  */
  double stim_t1;        /*   takes the current's exact average over the step            */
  int qoi;               /* mlmc_qoi: the nodal quantity the estimators average          */
  /* The paper's own KL variant (Sec. 3.1.1, Eq. KL-expansion-deterministic;
     Sec. 4): kl_kind = MLMC_KL_AFFINE_GAUSSIAN selects it; zero keeps the
     separable exponential kernel above. */
  int kl_kind;           /* mlmc_kl_kind                                                 */
  double kl_tol;         /* pivoted Cholesky stops at a remainder trace <= kl_tol x trace */
  double kl_s;           /* s of G = G0 (1 + s Z), capped by the ellipticity rule:        */
  double kl_delta;       /*   s_eff = min(kl_s, kl_delta / max_x sum_k |l_k(x)|)         */
  int kl_cand_n[3];      /* cells per axis of the grid whose cell centroids are the pivot
                            candidates (zeros: level 0's grid); independent of the levels,
                            so that contexts of different hierarchies share one field    */
} mlmc_config;

/* Random field of the conductivity.
 * MLMC_KL_SEPARABLE_EXP: s_l = s_l0 exp(Z), Z = sum_k sqrt(lam_k) phi_k xi_k,
 *   the analytic eigenpairs of kl_sigma2 exp(-|dx|/ell - |dy|/ell (- |dz|/ell)),
 *   xi_k ~ N(0, 1); conductivity tensor s_t I + (s_l - s_t) f f^T.
 * MLMC_KL_AFFINE_GAUSSIAN: the paper's G = s_l0 (1 + s_eff Z) I (isotropic),
 *   Z = sum_k l_k(x) y_k, y_k ~ U(-1, 1) (from the same Philox words: 2u - 1),
 *   l_k the columns of the pivoted Cholesky factor (Harbrecht, Peters &
 *   Schneider 2012) of kl_sigma2 exp(-|x - x'|^2 / kl_ell^2) over the cell
 *   centroids of the kl_cand_n grid (at most kl_modes columns, fewer when the
 *   remainder trace falls to kl_tol of the trace), extended to every level's
 *   centroids by the factor's own recursion (Nystrom), so that both members of
 *   a pair see the same continuous field; s_eff keeps G within
 *   s_l0 (1 +- kl_delta) for every y. */
typedef enum {
  MLMC_KL_SEPARABLE_EXP = 0,
  MLMC_KL_AFFINE_GAUSSIAN = 1
} mlmc_kl_kind;

/* Time scheme of the space-time blocks (block row k divided by dt):
 *   F_k(u) = (M/dt)(u_k - u_{k-1}) + K (theta u_k + (1-theta) u_{k-1})
 *            - M r(u_k) - M s_k,
 * theta = 1 implicit Euler (A = M/dt + K, B = -M/dt), theta = 1/2 the
 * Crank-Nicolson blocks of Sec. 3.2 (A = M/dt + K/2, B = -M/dt + K/2), the
 * reaction r(u) = c u(1-u)(u-a) at the new time level as in Eq. mono_disc. */
typedef enum {
  MLMC_SCHEME_IE = 0,
  MLMC_SCHEME_CN = 1
} mlmc_scheme;

typedef enum {
  MLMC_STIM_BALL = 0,    /* u(x, 0) = 1 for |x - stim_c| < stim_r, else 0          */
  MLMC_STIM_PULSE = 1    /* u(x, 0) = 0 and the Gaussian applied-current pulse      */
} mlmc_stimulus;

typedef enum {
  MLMC_QOI_ACTIVATION = 0,   /* first t with u >= 1/2, linear in t (T if never)   */
  MLMC_QOI_FINAL_STATE = 1   /* u(x, T), the paper's plotted quantity (Sec. 4)     */
} mlmc_qoi;

/* Row a7 -- preconditioner of the Newton steps' CG (the paper's Krylov solver
 * is preconditioned by ILU / block Jacobi on CPUs, Sec. 3.5).
 * MLMC_PRECOND_JACOBI: z = r / |H_ii|.
 * MLMC_PRECOND_GMG: one symmetric geometric-multigrid V-cycle on
 *   K + diag(|M (1/dt - r'(u))|) over vertex-nested coarsenings of the level's
 *   grid (every even cell count halved while the grid has more than 512 nodes):
 *   linear interpolation P, restriction P^T, Galerkin coarse stiffness P^T K P,
 *   lumped coarse diagonal P^T d, l1-Jacobi smoothing (mg_nu sweeps before and
 *   after, mg_coarse_sweeps on the coarsest grid), in the CG's precision (FP32
 *   in MLMC_PREC_MIXED).  It is used on levels whose step Hessians are
 *   positive definite for every state (c dt max r' < 1, max r' =
 *   c((1+a)^2/3 - a)), where the Newton direction and so the selected root do
 *   not depend on the preconditioner; other levels keep Jacobi.  It runs in
 *   the global-memory cluster layout (layout codes 100 + C), which the
 *   automatic layout choice then selects. */
typedef enum {
  MLMC_PRECOND_JACOBI = 0,
  MLMC_PRECOND_GMG = 1
} mlmc_precond;

typedef enum {
  MLMC_SOLVER_AUTO = 0,    /* cluster layout where a sample fits, else block layout      */
  MLMC_SOLVER_BLOCK = 1,   /* one thread block per sample, vectors in global memory      */
  MLMC_SOLVER_CLUSTER = 2  /* one thread-block cluster per sample, vectors in shared memory */
} mlmc_solver;

/* Per-sample solver report, written by the solve calls (device array). */
typedef struct {
  int32_t status;        /* MLMC_OK or MLMC_ERR_NOT_CONVERGED                        */
  int32_t failed_step;   /* first step that did not converge (0 if none)             */
  int32_t newton_iters;  /* nonlinear iterations summed over the time steps          */
  int32_t cg_iters;      /* summed over all Newton steps                             */
  int32_t truncations;   /* CG runs stopped at negative curvature                    */
  int32_t halvings;      /* line-search step halvings, or retried pseudo-steps of the
                            gradient-flow continuation                              */
  int32_t max_newton;    /* largest Newton count of one step                         */
  int32_t pad;
} mlmc_sample_info;

typedef struct mlmc_ctx mlmc_ctx;

/* Create a context for one configuration on the current CUDA device.
 * Builds the KL mode table (Sec. 3.1.1, Eq. KL-expansion-deterministic) on the
 * host and copies it and the level descriptors to the device (small, owned by
 * the context).  *out is NULL on failure. */
mlmc_status mlmc_create(const mlmc_config* cfg, mlmc_ctx** out);
void mlmc_destroy(mlmc_ctx* ctx);
/* Description of the last failure of this context (or of mlmc_create when ctx
 * is NULL); never NULL. */
const char* mlmc_last_error(const mlmc_ctx* ctx);

/* Sizes of level l: nodes, cells and time steps (host outputs, any may be NULL). */
mlmc_status mlmc_level_info(const mlmc_ctx* ctx, int level, int64_t* nodes, int64_t* cells,
                            int32_t* steps);

/* Bytes of device workspace needed by mlmc_solve / mlmc_sample_level for n
 * samples of level l (256-byte aligned pointer required). */
mlmc_status mlmc_workspace_bytes(const mlmc_ctx* ctx, int level, int n, size_t* bytes);

/* Row a1 -- xi for n samples (Sec. 3.1.1: the psi_k / y_k of the KL expansion,
 * here standard normal): Philox4x32-10 (Salmon et al., SC'11) with
 *   counter = (mode pair j, lo32(id), hi32(id), level), key = (lo32(seed), hi32(seed)),
 * and Box-Muller with correctly rounded operations only, so that the values
 * are bit-reproducible.  ids: device [n]; xi: device [n][kl_modes]. */
mlmc_status mlmc_xi(mlmc_ctx* ctx, uint64_t seed, int level, const uint64_t* ids, int n,
                    double* xi, void* stream);

/* Row a2 -- truncated KL field on the cell centroids of grid level l
 * (Sec. 3.1.1, Eq. KL-expansion-deterministic):
 *   Z[s][cell] = sum_k sqrt(lam_k) phi_k(centroid) xi[s][k].
 * xi: device [n][kl_modes]; Z: device [n][cells_l]. */
mlmc_status mlmc_kl_field(mlmc_ctx* ctx, int level, const double* xi, int n, double* Z,
                          void* stream);

/* Row a2, mixed precision -- the same field as mlmc_kl_field computed as one
 * dense contraction (cells x modes) . (modes x samples) on the tensor cores
 * (tcgen05 kind::tf32, accumulators in tensor memory) with the three-term
 * split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi of FP32 operands into TF32
 * parts: FP32 accuracy (|error| <~ 1e-6 max|Z|), FP64 output.  xi, n, Z as
 * for mlmc_kl_field (n <= 65535 * 256); ws: device workspace of
 * mlmc_kl_tc_workspace_bytes(ctx, n) bytes, 256-byte aligned (the split
 * sample operand, written and read by the call).  MLMC_PREC_MIXED pipelines
 * use it on the levels whose inner solves run in FP32; the others use
 * mlmc_kl_field.  A tile whose bounded wait for the tensor cores runs out
 * leaves its outputs unwritten and is reported by the next mlmc_run /
 * mlmc_run_more as MLMC_ERR_TIMEOUT. */
mlmc_status mlmc_kl_tc_workspace_bytes(const mlmc_ctx* ctx, int n, size_t* bytes);
/* The KL expansion's rank (kl_modes, or the pivoted Cholesky's rank) and, for
 * MLMC_KL_AFFINE_GAUSSIAN, the capped scale s_eff (1 otherwise); host outputs,
 * any may be NULL. */
mlmc_status mlmc_kl_info(const mlmc_ctx* ctx, int* rank, double* s_eff);
/* Check of the bounded-wait paths (the paper has no counterpart): with polls >=
 * 0, every tile of the context's later tensor-core KL launches first waits at
 * most `polls` polls on a barrier that nothing arms -- before it issues any
 * copy or MMA, so nothing is left in flight -- and takes its timeout exit
 * (outputs unwritten, counted; the next mlmc_run / mlmc_run_more reports
 * MLMC_ERR_TIMEOUT, and mlmc_reset clears the count); and the first barrier of
 * every group-layout solve waits, at most `polls` polls, for one CTA more than
 * the group has, so that each of its samples ends with status MLMC_ERR_TIMEOUT
 * in its mlmc_sample_info.  polls = -1 restores normal operation.  The device
 * and the context stay usable throughout. */
mlmc_status mlmc_check_timeout_path(mlmc_ctx* ctx, long long polls);
mlmc_status mlmc_kl_field_tc(mlmc_ctx* ctx, int level, const double* xi, int n, double* Z,
                             void* ws, size_t ws_bytes, void* stream);

/* Rows a3-a8 -- per-sample solve on grid level l: conductivity from Z, Q1
 * assembly, implicit Euler over all m_l steps with Newton (Sec. 3.3, 3.5),
 * activation times.
 *   Z:      device [n][cells_l]            (input)
 *   t_act:  device [n][nodes_l]            (output; T where never activated)
 *   slab:   device [n][m_l + 1][nodes_l] or NULL (output: every time slice)
 *   info:   device [n] or NULL             (output)
 *   ws:     device workspace of mlmc_workspace_bytes(ctx, l, n) bytes.
 * A sample that does not converge is reported in info[s].status and does not
 * affect the others. */
mlmc_status mlmc_solve(mlmc_ctx* ctx, int level, const double* Z, int n, double* t_act,
                       double* slab, mlmc_sample_info* info, void* ws, size_t ws_bytes,
                       void* stream);

/* Row a4 over the whole slab -- the all-at-once space-time residual of
 * Eq. mono_disc (implicit-Euler blocks), one launch for all n samples:
 *   F[s][k-1] = (M/dt)(u_k - u_{k-1}) + K u_k - M c u_k(1-u_k)(u_k-a),  k = 1..m_l
 *   res_max[s] = max_{k,i} |F[s][k-1][i]| / M_i.
 * slab: device [n][m_l+1][nodes_l]; Z as for mlmc_solve; F: device
 * [n][m_l][nodes_l] or NULL; res_max: device [n] or NULL. */
mlmc_status mlmc_slab_residual(mlmc_ctx* ctx, int level, const double* Z, const double* slab,
                               int n, double* F, double* res_max, void* stream);

/* Row a8 -- activation times from a stored slab (first crossing of 1/2,
 * linear in time; 0 where u_0 >= 1/2; T where never crossed).
 * slab: device [n][m_l+1][nodes_l]; t_act: device [n][nodes_l]. */
mlmc_status mlmc_activation(mlmc_ctx* ctx, int level, const double* slab, int n, double* t_act,
                            void* stream);

/* Rows a1-a9 -- n level-l sample pairs (Sec. 3.1.2, Eq. MLMC-estimator): one xi
 * per pair (counter level = l), the fine (l) and coarse (l-1) problems solved
 * with that xi, activation maps injected onto the level-0 vertices and
 *   y[s]  = t_l - t_{l-1},   y2[s] = t_l^2 - t_{l-1}^2     (t_{-1} = 0).
 * ids: device [n]; y, y2: device [n][nodes_0]; t_fine: device [n][nodes_l] or
 * NULL; t_coarse: device [n][nodes_{l-1}] or NULL; info: device [2n] or NULL
 * (fine reports first, then coarse); ws: mlmc_workspace_bytes(ctx, l, n). */
mlmc_status mlmc_sample_level(mlmc_ctx* ctx, int level, uint64_t seed, const uint64_t* ids,
                              int n, double* y, double* y2, double* t_fine, double* t_coarse,
                              mlmc_sample_info* info, void* ws, size_t ws_bytes, void* stream);

/* Row a10 -- merge a batch of n pair differences into the context's per-level
 * running estimates (Welford / Chan et al. pairwise update, FP64, fixed order).
 * y, y2: device [n][nodes_0]. */
mlmc_status mlmc_accumulate(mlmc_ctx* ctx, int level, const double* y, const double* y2, int n,
                            void* stream);
/* Clear every level's running estimates. */
mlmc_status mlmc_reset(mlmc_ctx* ctx, void* stream);

/* Row a10 -- the estimates (host outputs, any may be NULL; synchronises the
 * stream).  mean, var: [nodes_0] = sum_l mean(Y_l) and the second-moment
 * telescoping sum minus mean^2 (clipped at 0); mean_l, var_l: [n_levels][nodes_0];
 * V_l: [n_levels] = sum_i w_i Var(Y_l)_i with w the level-0 lumped mass;
 * N_l: [n_levels]; rmse: sqrt(sum V_l/N_l + bias^2), bias = ||mean(Y_L)||_w
 * (0 for one level). */
mlmc_status mlmc_estimate(mlmc_ctx* ctx, double* mean, double* var, double* mean_l,
                          double* var_l, double* V_l, int64_t* N_l, double* rmse, void* stream);

/* Autotuner for the solve kernel's layout on one level (the paper has no
 * counterpart; its solver runs on CPU clusters).  Layout codes: -1 the
 * block-per-sample kernel (global-memory vectors, one CTA per sample); 1, 2,
 * 4, 8, 16 a thread-block cluster of that many CTAs per sample with every
 * vector in shared memory (each CTA a band of whole rows; only where a band
 * fits); 100 + C (C = 1, 2, 4, 8, 16) a cluster of C CTAs per sample with the
 * vectors in global memory (the nodes dealt to the CTAs in chunks, cyclically);
 * 300 + C (C = 1, 2, 4, 8, 16) the same with 256-thread CTAs (twice as many
 * samples resident per SM);
 * MLMC_LAYOUT_GROUP (3D grids) G CTAs per sample that are not a hardware
 * cluster -- an ordinary grid whose CTAs form groups of G in arrival order and
 * synchronise through bounded global-memory barriers (a wait that runs out,
 * after 180 s, fails the sample with MLMC_ERR_TIMEOUT) -- with G = k SMs / n
 * for the largest k (CTAs per SM) that keeps G <= S/2 (S resident CTAs on the
 * device) and at least 1024 nodes per CTA (512 when the layout is set
 * explicitly), so that a few samples of a large grid use every SM, evenly,
 * instead of at most 16; a context runs its group
 * launches one after another, and at most two may run at once on one device;
 * 0 automatic: the smallest shared-memory cluster that holds a sample, else
 * (3D) the group layout where G >= 32, else global-memory clusters of up to 16
 * CTAs.  Each candidate (the block kernel only with
 * solver = MLMC_SOLVER_AUTO) solves the same n samples (ids device [n], drawn
 * with `seed`) once and is timed with CUDA events; the fastest becomes the
 * level's layout for every later solve of this context.
 * ws: mlmc_workspace_bytes(ctx, level, n).  Outputs (host, may be NULL): best
 * (its code) and ms [MLMC_TUNE_CANDIDATES] in the order -1, 1, 2, 4, 8, 16,
 * 101, 102, 104, 108, 116, 301, 302, 304, 308, MLMC_LAYOUT_GROUP (-1 where a
 * candidate was not run).  Synchronises the stream.  A forced cfg.cluster_size still wins over
 * the tuned value. */
#define MLMC_TUNE_CANDIDATES 16
#define MLMC_LAYOUT_GROUP 200
mlmc_status mlmc_autotune(mlmc_ctx* ctx, int level, uint64_t seed, const uint64_t* ids, int n,
                          void* ws, size_t ws_bytes, int* best, float* ms, void* stream);
/* The layout code used for a level, and a way to set it without tuning (e.g.
 * from a stored tuning result).  A shared-memory cluster size whose band does
 * not fit falls back to the automatic choice. */
mlmc_status mlmc_get_layout(const mlmc_ctx* ctx, int level, int* layout);
mlmc_status mlmc_set_layout(mlmc_ctx* ctx, int level, int layout);

/* Whole MLMC run with fixed sample counts (host N_l[n_levels]): for each level
 * l, sample ids 0..N_l-1 in batches of at most `batch` pairs, mlmc_sample_level
 * + mlmc_accumulate; then mlmc_estimate into the host outputs (as above;
 * synchronises the stream).  Resets the running estimates first.  Levels run
 * concurrently on streams owned by the context (ordered after the work already
 * on `stream`; `stream` waits for them); within a level the fine and coarse
 * solves of a batch run concurrently.  On a 3D level whose grids take the
 * group layout (see mlmc_autotune) a batch holds at most as many samples as
 * groups of >= 32 CTAs are resident at once (9 on a 152-SM device); the
 * workspace size accounts for it.  ws: mlmc_run_workspace_bytes(ctx, N_l,
 * batch) bytes.
 * C_l (host [n_levels], may be NULL): the cost C_l of Sec. 3 per pair of level
 * l, in seconds: device time of the solve-kernel launches of its fine and
 * coarse solves (CUDA events around each launch, summed) divided by N_l.
 * Levels and solves overlap on the device, so this is the cost of a pair
 * under the same sharing, not an exclusive one.
 * stats (host [9], may be NULL): device ms spent in the per-sample solve
 * kernel (CUDA events around its launches, summed), its launch count, CG and
 * Newton iterations summed over samples and weighted by the nodes of their
 * grid, CG truncations, line-search halvings, non-converged solves, the total
 * number of kernels launched, and the node-weighted CG iterations run in
 * FP64.  Returns MLMC_ERR_NOT_CONVERGED (outputs still written) if any solve
 * failed. */
mlmc_status mlmc_run(mlmc_ctx* ctx, const int64_t* N_l, uint64_t seed, int batch, void* ws,
                     size_t ws_bytes, double* mean, double* var, double* V_l, double* C_l,
                     double* rmse, double* stats, void* stream);
/* Per-level solve statistics (host out [n_levels][8]) of the solves on grid
 * level l (as the fine member of pair l or the coarse member of pair l+1):
 * out[8l + 0] the device ms of their solve-kernel launches in the last
 * mlmc_run / mlmc_run_more / mlmc_run_to_rmse round (CUDA events around each
 * launch, summed), [1] their number, and since the last reset: [2] CG iterations x
 * nodes, [3] nonlinear iterations x nodes, [4] the part of [2] run in FP64,
 * [5] CG truncations, [6] halvings or retried pseudo-steps, [7] solves that did
 * not converge.  Used to set each level's work against its own bound. */
mlmc_status mlmc_level_stats(mlmc_ctx* ctx, double* out);

/* Workspace bytes for mlmc_run with the given counts (host N_l) and batch;
 * also for mlmc_run_more with N_l = its count. */
mlmc_status mlmc_run_workspace_bytes(const mlmc_ctx* ctx, const int64_t* N_l, int batch,
                                     size_t* bytes);

/* Incremental run: adds count[l] level-l pairs with sample ids first_id[l] ..
 * first_id[l]+count[l]-1 (host arrays) to the running estimates, without a
 * reset, in the same concurrent schedule as mlmc_run.  Because every sample's
 * random input is a function of (seed, level, id) alone, splitting ids
 * 0..N-1 over several calls -- or several contexts, on several devices, whose
 * states are then merged with mlmc_merge_states -- gives the sample set of
 * one mlmc_run with N_l = N; the merged moments equal it up to the rounding
 * order of the accumulation.  solve_seconds (host [n_levels], may be NULL):
 * each level's summed solve-kernel device time.  Synchronises the stream.
 * ws: mlmc_run_workspace_bytes(ctx, count, batch).  Returns
 * MLMC_ERR_NOT_CONVERGED if any solve of this call failed. */
mlmc_status mlmc_run_more(mlmc_ctx* ctx, const int64_t* first_id, const int64_t* count,
                          uint64_t seed, int batch, void* ws, size_t ws_bytes,
                          double* solve_seconds, void* stream);

/* Adaptive MLMC with a fixed hierarchy (the sample allocation of Sec. 3.1.2,
 * with the error of Eq. general-error-MLMC split into sampling error and bias):
 * runs the pilot counts N_pilot[l] (>= 1 each), then up to max_rounds times
 * estimates V_l (lumped-mass-weighted variance of Y_l) and the cost C_l per
 * pair (solve-kernel seconds, as for mlmc_run) and raises every level to
 *   N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k)),
 * capped at max_per_level, running only the new ids.  This is the allocation
 * that makes the sampling error sum_l V_l / N_l at most eps^2 / 2 at least
 * total cost.  Stops when no level needs more samples.  Resets the running
 * estimates first.  Outputs (host): N_l [n_levels] samples used, mean, var
 * [nodes_0] (may be NULL), V_l, C_l [n_levels] (may be NULL), rmse (as
 * mlmc_estimate, sampling error plus squared bias) and bias (the weighted norm
 * of the finest level's mean correction, an estimate of the discretisation
 * bias; 0 for one level) (may be NULL).  The target RMSE <= eps also needs
 * bias^2 <= eps^2 / 2: when the bias estimate is larger, the call returns
 * MLMC_WARN_BIAS (outputs valid; mlmc_last_error says by how much) -- no
 * sample count can reach eps on this hierarchy, only finer levels can.  ws:
 * mlmc_run_workspace_bytes(ctx, {batch, ..., batch}, batch) bytes. */
mlmc_status mlmc_run_to_rmse(mlmc_ctx* ctx, double eps, const int64_t* N_pilot, int max_rounds,
                             int64_t max_per_level, uint64_t seed, int batch, void* ws,
                             size_t ws_bytes, int64_t* N_l, double* mean, double* var,
                             double* V_l, double* C_l, double* rmse, double* bias, void* stream);

/* Row a11 diagnostics of the running estimates (host outputs, any may be NULL;
 * synchronises the stream), for judging the bias of the hierarchy
 * (Sec. 3.1.2, Eq. discretization-error and Eq. general-error-MLMC):
 *   mean_norm [n_levels]: ||mean(Y_l)||_w, the level-0 lumped-mass-weighted L2
 *     norm of each level's mean correction (of the level-0 mean for l = 0);
 *   alpha: the fitted weak rate, the least-squares slope of
 *     -log2 ||mean(Y_l)||_w over the correction levels l >= 1 (NaN with fewer
 *     than two), so that the bias of level L is ~ ||mean(Y_L)|| 2^-alpha;
 *   censored [n_levels]: the fraction of the injected level-l activation times
 *     (every coarsest-grid node of every pair computed since the last reset)
 *     equal to T, i.e. nodes the front had not reached by the end time. */
mlmc_status mlmc_diagnostics(mlmc_ctx* ctx, double* mean_norm, double* alpha, double* censored,
                             void* stream);

/* Accumulator state (checkpoint / resume, and the cross-device merge).  The
 * state of a context is, per level l, the sample count N_l and per coarsest-
 * grid node the running mean and sum of squared deviations of the injected
 * difference Y_l and the running mean of t_l^2 - t_{l-1}^2: host arrays
 * N_l [n_levels] and mean_l, m2_l, mean2_l [n_levels][nodes_0] (row l at
 * offset l * nodes_0).  mlmc_get_state copies it out (any pointer may be
 * NULL; synchronises the stream); mlmc_set_state replaces it (all required).
 */
mlmc_status mlmc_get_state(mlmc_ctx* ctx, int64_t* N_l, double* mean_l, double* m2_l,
                           double* mean2_l, void* stream);
mlmc_status mlmc_set_state(mlmc_ctx* ctx, const int64_t* N_l, const double* mean_l,
                           const double* m2_l, const double* mean2_l, void* stream);
/* Host-only merge of state b into state a (same layout as above): for every
 * level the pairwise update of Chan, Golub and LeVeque (1979) for count,
 * mean and sum of squared deviations, and the count-weighted mean of mean2.
 * Runs on the CPU, needs no device or context; the single exchange step of a
 * multi-device run.  MLMC_ERR_ARG on NULL pointers or negative counts. */
mlmc_status mlmc_merge_states(int levels, int64_t nodes0, int64_t* N_a, double* mean_a,
                              double* m2_a, double* mean2_a, const int64_t* N_b,
                              const double* mean_b, const double* m2_b, const double* mean2_b);

/* ------------------------------------------------------------------ serving
 * Request server on one context (the paper has no counterpart; it is the
 * serving form of the method: MLMC sample requests arrive over time and the
 * running estimate is updated as they finish).  A request is one level pair
 * (level, seed, sample id) with an optional stimulus centre.  A native
 * scheduler thread admits queued requests as batches of one level whenever a
 * slot (a pair of streams) is free and a device arena of mem_budget bytes,
 * allocated once at creation, has room for the batch (a batch that does not
 * fit is halved until it does: memory-based admission).  Batches of different
 * levels run concurrently.  Finished batches are merged into the context's
 * running estimates (mlmc_accumulate order: completion order) and their
 * results are queued for mlmc_server_poll.  A request's result depends only on
 * the request, not on what else is in flight.  While a server exists, the
 * context must not be used directly.  Times are seconds on the server's
 * monotonic clock (0 at creation). */
typedef struct mlmc_server mlmc_server;

typedef struct {
  int max_batch;      /* most requests of one level in one launch, 1..65535 */
  int slots;          /* batches in flight at once, 1..16 */
  size_t mem_budget;  /* device bytes for in-flight batches (the arena) */
  int keep_maps;      /* nonzero: results carry the fine activation map */
  double max_wait_s;  /* hold a partial batch this long while the device is busy */
} mlmc_server_config;

typedef struct {
  int64_t tag;        /* caller's identifier, returned in the result */
  int level;          /* level pair, 0..n_levels-1 */
  int pad;
  uint64_t seed;      /* xi seed of this request (Philox key) */
  uint64_t sample_id; /* xi counter of this request */
  double stim_c[3];   /* stimulus centre; NaN in stim_c[0]: the configuration's */
} mlmc_request;

typedef struct {
  int64_t tag;
  int level;
  int status;         /* MLMC_OK, or the status of a failed solve */
  int newton_iters;   /* summed over the pair's solves */
  int cg_iters;
  double t_submit, t_admit, t_done;
} mlmc_result;

/* Creates the server and starts its scheduler thread.  MLMC_ERR_WORKSPACE if
 * mem_budget cannot hold one request of the largest level. */
mlmc_status mlmc_server_create(mlmc_ctx* ctx, const mlmc_server_config* cfg, mlmc_server** out);
/* Queues n requests (host array, copied); thread-safe, does not block on the
 * device.  MLMC_ERR_ARG for a level out of range (nothing queued). */
mlmc_status mlmc_server_submit(mlmc_server* s, const mlmc_request* reqs, int n);
/* Takes up to max finished results (host out[max]); waits up to timeout_s for
 * the first.  y (host [max][nodes_0] or NULL) receives each request's Y_l on
 * the coarsest grid; maps (host [max][map_stride] or NULL, keep_maps only) its
 * fine activation map (nodes of its level).  Thread-safe. */
mlmc_status mlmc_server_poll(mlmc_server* s, mlmc_result* out, int max, int* count, double* y,
                             double* maps, int64_t map_stride, double timeout_s);
/* Waits until every submitted request has finished (MLMC_ERR_TIMEOUT after
 * timeout_s). */
mlmc_status mlmc_server_drain(mlmc_server* s, double timeout_s);
/* stats (host [8]): submitted, queued, in flight, completed, batches launched,
 * largest queue length seen, peak arena bytes, sticky error status. */
mlmc_status mlmc_server_stats(mlmc_server* s, int64_t* stats);
mlmc_status mlmc_server_clock(mlmc_server* s, double* now);
/* The running MLMC estimate over the finished requests (as mlmc_estimate;
 * host outputs, any may be NULL; bias as in mlmc_run_to_rmse). */
mlmc_status mlmc_server_estimate(mlmc_server* s, double* mean, double* var, double* V_l,
                                 int64_t* N_l, double* rmse, double* bias);
const char* mlmc_server_error(mlmc_server* s);
/* Stops admitting, waits for the batches in flight, frees everything. */
void mlmc_server_destroy(mlmc_server* s);

/* Measurement aid (the paper has no counterpart): the device's fused
 * multiply-add rate in TFLOP/s (2 flop per FMA), FP64 (fp64 != 0) or FP32,
 * from 8 independent FMA chains per thread on 16 x 256 threads per SM, timed
 * with CUDA events on `stream` after a warm-up launch; synchronises it.  out:
 * device scratch of >= 16 * 256 * 8 bytes per SM (written).  This is the ALU
 * bound of the sweep's FP64 and FP32 work. */
mlmc_status mlmc_probe_fma_rate(int fp64, void* out, size_t out_bytes, double* tflops,
                                void* stream);

/* Allocation-free variant of mlmc_solve (the paper has no counterpart; this is
 * a deployment aid).  For callers that may not allocate device memory -- for
 * example code running under a host framework that reserved the whole device
 * budget up front, a plugin that must not touch the device heap, or a caller
 * that cannot afford the device-wide synchronisation an allocation may cause.
 * The caller passes only inputs and outputs, exactly as for mlmc_solve
 * (without the slab output): Z device [n][cells_l], t_act device [n][nodes_l],
 * info device [n] or NULL, plus the configuration itself (no context needed).
 *
 * Scratch: one file-scope device array of MLMC_NOALLOC_SCRATCH_BYTES bytes,
 * held by every device that uses it until the process exits.  The call
 * allocates nothing (no cudaMalloc/cudaFree, no allocating library routine).
 * Requests whose scratch would exceed the array are rejected with
 * MLMC_ERR_WORKSPACE and a message naming both sizes (read it with
 * mlmc_last_error(NULL)); other failures set the same message.
 * Set-up: the first call on a device (with that device current) looks up the
 * array's device address and loads the modules of the kernels it launches,
 * once per device, under a lock.  CUDA loads modules lazily by default, so it
 * is this first call -- not the loading of the library -- that places the
 * 16 MiB array and the kernels' code on the device.  Make that first call
 * during the caller's own set-up (a call with n = 1 is enough), before any
 * stream capture and while device memory can still be committed; later calls
 * only enqueue the assembly and the sweep.
 * Every call on a device shares the one array and leaves its contents behind;
 * the solve writes every scratch word before reading it, so nothing needs
 * clearing, but calls whose work overlaps on the GPU (other streams, other
 * host threads) race on the scratch and must be serialised by the caller.
 * The level geometry, precision rule and solver parameters are derived from
 * cfg exactly as mlmc_create and mlmc_solve derive them; a level whose grid
 * exceeds 2^31 nodes or 2^20 cells per axis is rejected with MLMC_ERR_ARG. */
#define MLMC_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
mlmc_status mlmc_solve_noalloc(const mlmc_config* cfg, int level, const double* Z, int n,
                               double* t_act, mlmc_sample_info* info, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MLMC_H */
