// Internal definitions shared by the CUDA translation units of the library.
// Everything here is device-side layout and launch plumbing; the arithmetic of
// each step lives in its own file (rng.cu, kl.cu, assemble.cu, solver.cu,
// slab.cu, estimators.cu) and the C ABI in abi.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mlmc.h"

namespace mlmc {

// Geometry of one grid level (Q1 nodes on a box, x fastest).
struct LevelDesc {
  int dim;
  int n[3];        // cells per axis (1 on unused axes)
  int N[3];        // nodes per axis (1 on unused axes)
  int m;           // implicit-Euler steps
  int64_t nodes, cells;
  double h[3];     // cell sides (1 on unused axes)
  double vol;      // cell volume (area in 2D)
  double dt, T;
};

// Physical parameters copied by value into kernels.
struct Physics {
  double c, a, s_t, s_l0;
  double th0, th1;       // fiber angle (radians) at z = 0 and z = L[2]
  double Lz;
  double stim_r2;        // squared stimulus radius
  double stim_c[3];
  const double* stim_ps; // per-sample stimulus centres, device [n][3], or NULL
  // time scheme: theta = 1 implicit Euler, 1/2 Crank-Nicolson (the couplings
  // are assembled times theta; the residual adds (1-theta)/theta times the
  // scaled stencil of u_{k-1})
  double theta;
  // stimulus kind 1: u0 = 0 and the applied current amp exp(-|x - c|^2 isig2)
  // on 0 <= t < t1 (kind 0: u0 = 1 in the ball of radius sqrt(stim_r2))
  int stim_kind;
  double stim_amp, stim_isig2, stim_t1;
  int qoi;               // 0: activation time; 1: the final state u(T)
  int cond_kind;         // 0: fiber tensor, s_l = s_l0 exp(Z); 1: isotropic s_l0 (1 + Z)
};

// The applied current averaged over step k (1-based) at squared distance r2
// from the centre: amp exp(-r2 isig2) |[t_{k-1}, t_k] ∩ [0, t1)| / dt.
__host__ __device__ inline double stim_step_scale(const Physics& p, int k, double dt) {
  if (p.stim_kind != 1) return 0.0;
  const double a = (k - 1) * dt, b = k * dt;
  const double ov = (b < p.stim_t1 ? b : p.stim_t1) - a;
  return ov > 0.0 ? p.stim_amp * ov / dt : 0.0;
}

struct SolverParams {
  double newton_tol;
  int newton_max;
  double lin_rtol;
  int lin_max;
  double ls_full_step;   // max|d| below which the full Newton step is taken
  int flow;              // the level's steps have several roots (c dt max r' > 1):
                         // gradient-flow continuation instead of Newton-CG
  double tau0;           // first pseudo-step of the continuation, 1 / (2 max r')
  int cg_scale;          // FP32 CG: solve for a power-of-two scaled right-hand side
  int pred_stencil = 1;       // global-memory layouts: the predicated branch-free stencil
                              // for every node (1), or the constant-offset stencil for
                              // interior nodes and the bounds-checked one at the boundary
  long long grp_check = -1;   // >= 0: check of the group layout's bounded waits -- the
                              // first barrier waits for one arrival too many, at most
                              // grp_check polls, and the sample ends with MLMC_ERR_TIMEOUT
};

// Gradient-flow continuation (levels with c dt max r' > 1; max r' =
// c((1+a)^2/3 - a)).  Such a step has several roots; the root is the end
// point of the gradient flow M v' = -F(v) of the step energy from u_{k-1},
// the local minimum in whose basin u_{k-1} lies.  It is reached by linearly
// implicit pseudo-steps (M/t + H(u)) d = -F(u): t starts at tau0; a step whose
// CG meets non-positive curvature (M/t + H not positive definite) is retried
// with t/4 -- with M/t + H positive definite a step never reverses the flow's
// unstable component near a saddle; a step moving a node by more than
// FLOW_MOVE is taken shortened to that move (a positive multiple of the same
// direction) and the next t shrinks accordingly, otherwise t grows towards the
// move limit, at most doubling; once an accepted step moves no node by more
// than the switch threshold (FLOW_NEWTON at first) Newton steps finish the
// solve while their CG meets only positive curvature and they move no node by
// more than 10x the threshold (else the flow resumes with a 10x smaller
// threshold).
constexpr double FLOW_MOVE = 0.3;
constexpr double FLOW_TMIN = 1e-9;
constexpr double FLOW_TMAX = 1e20;
constexpr double FLOW_NEWTON = 1e-2;
inline bool level_has_several_roots(double c, double a, double dt) {
  return dt * c * ((1.0 + a) * (1.0 + a) / 3.0 - a) > 1.0;
}

// Configuration-derived quantities shared by mlmc_create, mlmc_solve and
// mlmc_solve_noalloc (defined in abi.cu).
bool derive_level(const mlmc_config& c, int level, LevelDesc* lv, std::string* err);
bool model_config_ok(const mlmc_config& c);
void derive_physics(const mlmc_config& c, Physics* ph);
// FP32 inner solves are used only where the step Jacobian is at most mildly
// indefinite: MLMC_PREC_MIXED and c dt max r' <= mixed_cdr_max (default 2).
bool level_mixed(const mlmc_config& c, const LevelDesc& lv);
SolverParams level_solver_params(const mlmc_config& c, const LevelDesc& lv, bool mixed);
// Byte offsets of one level's solver scratch for n samples (the workspace of
// mlmc_solve), 256-byte aligned.
struct SolveWs {
  size_t coef64, coef32, ubuf, F, Ku, Kd, kr, mg, grp, total;
};
SolveWs solve_ws(const mlmc_config& c, const LevelDesc& lv, int n, bool mixed);

// FP32 inner solves on grids whose lumped mass per time step is this small
// (the fine 3D levels) scale the CG's right-hand side by a power of two: their
// late Newton residuals otherwise push the CG's r.z below FP32's normal range.
inline bool cg_needs_scaling(const LevelDesc& lv) { return lv.vol / lv.dt < 1e-4; }

// Geometric multigrid hierarchy of one grid level (the CG preconditioner of
// the global-memory cluster layout).  Level 0 is the level's own grid; level
// g+1 halves every axis of level g whose cell count is even (vertex-nested, so
// coarse node I sits on fine node 2I).  Per sample the workspace holds, in the
// CG's precision, at element offsets relative to the sample's block:
//   level 0: ks (row sums of |K|), xa, xb (smoother ping-pong), t (residual);
//   level g >= 1: K [3^dim][nodes] (Galerkin couplings), ks, d (lumped
//   diagonal term), inv (l1-Jacobi inverse), xa, xb, b (right-hand side), t.
constexpr int MG_MAX_LEVELS = 10;
struct MGLevel {
  int n[3];           // cells per axis
  int N[3];           // nodes per axis
  int nodes;
  int cz[3];          // 1: axis halved from this level to the next
  int64_t K, ks, d, inv, xa, xb, b, t;   // element offsets (K, d, inv, b unused on level 0)
};
struct MGDesc {
  int G;              // levels (G = 0: no multigrid)
  int nu;             // pre- and post-smoothing sweeps
  int coarse_sweeps;  // l1-Jacobi sweeps on the coarsest level
  int64_t per_sample; // elements per sample
  MGLevel l[MG_MAX_LEVELS];
};
// Builds the hierarchy of grid lv: coarsen while some axis has an even cell
// count and the grid has more than 512 nodes.
void mg_hierarchy(const LevelDesc& lv, int nu, int coarse_sweeps, MGDesc* mg);

// Number of stencil couplings per node (3^dim) and the centre index.
__host__ __device__ inline int n_offsets(int dim) { return dim == 3 ? 27 : (dim == 2 ? 9 : 3); }
__host__ __device__ inline int centre_offset(int dim) { return dim == 3 ? 13 : (dim == 2 ? 4 : 1); }

// Lumped Q1 mass of node (i,j,k): cell volume times 1/2 per axis on which the
// node lies on the boundary (the row sum of the consistent mass).
__device__ inline double lumped_mass(const LevelDesc& lv, int i, int j, int k) {
  double m = lv.vol;
  if (i == 0 || i == lv.n[0]) m *= 0.5;
  if (lv.dim >= 2 && (j == 0 || j == lv.n[1])) m *= 0.5;
  if (lv.dim == 3 && (k == 0 || k == lv.n[2])) m *= 0.5;
  return m;
}

__device__ inline void node_ijk(const LevelDesc& lv, int64_t A, int& i, int& j, int& k) {
  i = (int)(A % lv.N[0]);
  int64_t r = A / lv.N[0];
  j = (int)(r % lv.N[1]);
  k = (int)(r / lv.N[1]);
}

// Spatial shape of the applied current at node (i, j, k): exp(-|x - c|^2 isig2),
// c the (per-sample) stimulus centre sc.
__device__ inline double stim_shape(const Physics& p, const LevelDesc& lv, const double* sc, int i,
                                    int j, int k) {
  const double x[3] = {i * lv.h[0], j * lv.h[1], k * lv.h[2]};
  double r2 = 0.0;
  for (int d = 0; d < lv.dim; ++d) r2 += (x[d] - sc[d]) * (x[d] - sc[d]);
  return exp(-r2 * p.stim_isig2);
}

// Reaction r(u) = c u (1-u)(u-a) and its derivative.
__device__ inline double rxn(const Physics& p, double u) { return p.c * u * (1.0 - u) * (u - p.a); }
__device__ inline double rxn_d(const Physics& p, double u) {
  return p.c * (-3.0 * u * u + 2.0 * (1.0 + p.a) * u - p.a);
}

// Kernels and launchers (defined in the .cu files).
cudaError_t launch_xi(uint64_t seed, const uint64_t* seeds, int level, const uint64_t* ids, int n,
                      int M, int uniform, double* xi, cudaStream_t st);
// The paper's KL variant (kl_affine.cu).  Host: pivoted Cholesky of the
// Gaussian covariance sigma2 exp(-|x - x'|^2 / ell^2) on the cell centroids of
// an n[3] grid (at most M columns; stop at a remainder trace <= tol of the
// full trace): the pivot coordinates xp [m][3] and the pivot rows of the
// factor lpiv [M][M]; *bound = max over the candidates of sum_k |L_ck| (the
// ellipticity rule's sup); returns the rank m.
int pivoted_cholesky_host(int dim, const double* L, const int* n, double sigma2, double ell, int M,
                          double tol, std::vector<double>& xp, std::vector<double>& lpiv,
                          double* bound);
// Device: the factor's columns at the cell centroids of lv (Nystrom
// extension), phi64 [cells][M] and phi32 (same in FP32, may be NULL); bound
// (device, may be NULL): the largest sum_k |phi_k| over the cells (atomic max
// on the bits of a non-negative double; zero it first).
cudaError_t launch_pc_eval(const LevelDesc& lv, int M, int m, double sigma2, double ell,
                           const double* xp, const double* lpiv, double* phi64, float* phi32,
                           unsigned long long* bound, cudaStream_t st);
// Z[s][cell] = sum_k phi64[cell][k] coef[k] xi[s][k] (FP64), the affine field.
cudaError_t launch_kl_field_table(const LevelDesc& lv, int M, const double* coef,
                                  const double* phi64, const double* xi, int n, double* Z,
                                  cudaStream_t st);
cudaError_t launch_kl_field(const LevelDesc& lv, int M, const double* sqrt_lam, const int* idx,
                            const double* phi_x, const double* phi_y, const double* phi_z,
                            int n1d, const double* xi, int n, double* Z, cudaStream_t st);
// Mixed-precision KL synthesis on the tensor cores (kl_tc.cu): three-term
// split-TF32 products, FP32 accumulation in tensor memory, FP64 output.  err
// (device) counts CTAs whose bounded wait for the tensor cores ran out.
// ws: kl_tc_workspace_bytes(M, n) bytes (the prepared B operand), 256-byte
// aligned; phi_*: the 1D mode tables in FP32.  check_limit >= 0 (a check of
// the timeout path): every CTA first waits at most that many polls on a
// barrier nothing arms, before issuing any copy or MMA, and takes its timeout
// exit; -1 for normal operation.
size_t kl_tc_workspace_bytes(int M, int n);
// phi_cells (FP32 [cells][M], or NULL): an explicit mode table instead of the
// separable 1D tables (the paper's KL variant).
cudaError_t launch_kl_field_tc(const LevelDesc& lv, int M, const double* sqrt_lam, const int* idx,
                               const float* phi_x, const float* phi_y, const float* phi_z,
                               const float* phi_cells, const double* xi, int n, double* Z, void* ws,
                               unsigned long long* err, long long check_limit, cudaStream_t st);
cudaError_t preload_kl_tc();
// sym (3D only): store each symmetric pair once -- per sample [14][nodes], the
// offsets 13..26 of {-1,0,1}^3 (centre first); the coupling to offset o < 13
// is the neighbour's entry 26 - o (the global-memory sweeps of 3D grids).
// The assembly is exactly symmetric (each pair sums the same cells in the same
// order), so both layouts hold the same numbers.
cudaError_t launch_assemble(const LevelDesc& lv, const Physics& ph, const double* Z, int n,
                            double* coef64, float* coef32, cudaStream_t st, bool sym = false);
// Loads the assembly kernels' module (both dimensions) without launching.
cudaError_t preload_assemble();
cudaError_t launch_solve(const LevelDesc& lv, const Physics& ph, const SolverParams& sp,
                         bool mixed, int n, const double* coef64, const float* coef32,
                         double* slab, double* ubuf, double* F, double* Ku, double* Kd,
                         void* kr, double* t_act, mlmc_sample_info* info,
                         unsigned long long* counters, cudaStream_t st);
// Cluster solver (solver_cluster.cu): C CTAs per sample, bands of H rows,
// nt threads per CTA, couplings in shared memory or not, smem bytes per CTA.
struct ClusterPlan {
  int C, H, nt;
  bool coef_smem;
  bool gm;        // vectors in global memory (H = nodes per CTA), else shared (H = rows per CTA)
  size_t smem;
  int G = 0;      // > 0: the group layout -- gm vectors, C = G CTAs per sample as a plain grid
};
// Group layout: per launch a ticket counter and per sample an arrival counter
// and a give-up flag (128 bytes apart), and the reductions' CTA partials
// [2][8][G] per sample.  GROUP_MAX_CTAS bounds G; the group area of a solve
// workspace holds GROUP_MAX_SAMPLES samples (launches with more samples use
// the cluster layouts).
constexpr int GROUP_MAX_CTAS = 1024;
constexpr int GROUP_MAX_SAMPLES = 64;
constexpr int GROUP_MAX_GRID = 4096;   // bound on samples x G of one launch
inline size_t group_sync_bytes(int n) { return (size_t)32 * 4 * (size_t)(n + 1); }
inline size_t group_slot_bytes(int n, int G) { return (size_t)n * 16 * (size_t)G * 8; }
// Global-memory vectors of the gm layout, per sample: u [2N], F [N] (FP64),
// r z p q d diag diag^-1 [7N] in the CG's precision, node codes [N].
struct ClusterGlobal {
  double* u = nullptr;
  double* F = nullptr;
  void* kr = nullptr;
  unsigned* code = nullptr;
  void* mg = nullptr;     // multigrid workspace (MGDesc::per_sample elements per sample), or NULL
  unsigned* gsync = nullptr;   // group layout: group_sync_bytes(n)
  double* gslot = nullptr;     // group layout: group_slot_bytes(n, G)
};
bool cluster_plan(const LevelDesc& lv, bool mixed, int want_C, ClusterPlan* plan, bool gm = false,
                  int nt = 512);
// Group layout plan for n samples of the 3D grid lv: G = k SMs / n CTAs per
// sample for the largest k (CTAs per SM) with G <= S / 2 (S the device's
// resident-CTA capacity for the group kernel), G <= GROUP_MAX_CTAS, n G <=
// GROUP_MAX_GRID and at least 1024 nodes per CTA (512 with force, the layout
// requested by code; where no such G exists it takes min(S / n, nodes / 512)).
// *ok = false when the layout does not apply: not 3D, n
// above GROUP_MAX_SAMPLES, or G below 32 (below 1 with force), where clusters
// of 16 CTAs serve as well.  G <= S / 2 keeps two group launches running at
// once (e.g. from two contexts) free of deadlock: each waits at most for one
// incomplete group of its own.
cudaError_t group_plan(const LevelDesc& lv, bool mixed, int n, bool force, ClusterPlan* plan, bool* ok);
// Samples of the 3D grid lv whose groups of at least 32 CTAs are resident at
// once (resident CTAs / 32; 0 when lv is not 3D).
cudaError_t group_resident_samples(const LevelDesc& lv, bool mixed, int* m);
size_t cluster_smem_bytes(int dim, int nmax, bool mixed, bool coef_smem, int nt);
// Loads the kernel instance a plan launches and sets its attributes, so that
// a timed launch does not include module loading.
cudaError_t preload_solve_cluster(const LevelDesc& lv, bool mixed, const ClusterPlan& pl);
cudaError_t preload_solve(const LevelDesc& lv, bool mixed);
// How many clusters of a plan can be resident at once on this device (0: the
// plan cannot launch here).
cudaError_t cluster_max_active(const LevelDesc& lv, bool mixed, const ClusterPlan& pl, int* count);
// mg: the multigrid hierarchy of lv (G > 0 and a gm plan: GMG-preconditioned
// CG; otherwise Jacobi).
cudaError_t launch_solve_cluster(const LevelDesc& lv, const Physics& ph, const SolverParams& sp,
                                 bool mixed, const ClusterPlan& pl, int n, const double* coef64,
                                 const float* coef32, double* slab, double* t_act,
                                 mlmc_sample_info* info, unsigned long long* counters,
                                 const ClusterGlobal& g, const MGDesc& mg, cudaStream_t st);
// counters (device, may be NULL) of one solve launch: [0] non-converged
// solves, [1] CG iterations x nodes, [2] nonlinear iterations x nodes, [3] CG
// truncations, [4] halvings / retried pseudo-steps, [5] CG iterations x nodes
// run in FP64 (the others run in FP32).  A context keeps one such block of
// CNT_PER_LEVEL counters per level at CNT_LEVEL + CNT_PER_LEVEL l, after its
// global counters: [6] tensor-core KL tiles whose bounded wait ran out,
// [7 + l] injected level-l activation times equal to T (censored).
constexpr int CNT_TC_TIMEOUT = 6;
constexpr int CNT_CENSORED = 7;
constexpr int CNT_LEVEL = CNT_CENSORED + MLMC_MAX_LEVELS;
constexpr int CNT_PER_LEVEL = 8;
constexpr int N_COUNTERS = CNT_LEVEL + CNT_PER_LEVEL * MLMC_MAX_LEVELS;
cudaError_t launch_slab_residual(const LevelDesc& lv, const Physics& ph, const double* coef64,
                                 const double* slab, int n, double* F, double* res_max,
                                 cudaStream_t st);
cudaError_t launch_activation(const LevelDesc& lv, const double* slab, int n, double* t_act,
                              cudaStream_t st);
// cens (device, may be NULL): incremented by the number of injected fine
// activation times equal to T (censored).
cudaError_t launch_pair_diff(const LevelDesc& l0, const LevelDesc& lf, const LevelDesc* lc,
                             const double* tf, const double* tc, int n, double* y, double* y2,
                             unsigned long long* cens, cudaStream_t st);
cudaError_t launch_accumulate(int64_t nodes0, const double* y, const double* y2, int n,
                              int64_t n_old, double* mean, double* m2, double* mean2,
                              cudaStream_t st);
cudaError_t launch_estimate(int levels, int64_t nodes0, const LevelDesc& l0, const int64_t* N_l,
                            const double* mean_l, const double* m2_l, const double* mean2_l,
                            double* out, cudaStream_t st);

}  // namespace mlmc
