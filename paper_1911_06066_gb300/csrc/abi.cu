// The C ABI (include/mlmc.h): argument checking, workspace carving, and the
// host-side orchestration of the per-level pipeline.  No arithmetic of the
// method runs here except the KL mode table (built once per context).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "ctx.cuh"

namespace mlmc {
void kl_1d_host(double len, double ell, int n, std::vector<double>& omega, std::vector<double>& lam,
                std::vector<double>& nrm);
bool kl_table_host(int dim, const double* L, double sigma2, double ell, int M, std::vector<int>& idx,
                   std::vector<double>& sqrt_lam);
void kl_phi_table_host(double len, double ell, int n1d, int n_axis, std::vector<double>& out);
cudaError_t launch_iota(uint64_t first, int n, uint64_t* ids, cudaStream_t st);
}  // namespace mlmc

using namespace mlmc;


static thread_local std::string g_create_error;

namespace mlmc {
// Message for mlmc_last_error(NULL) from entry points that take no context.
void set_create_error(const std::string& msg) { g_create_error = msg; }
}  // namespace mlmc

mlmc_status mlmc::fail(mlmc_ctx* ctx, mlmc_status st, const std::string& msg) {
  if (ctx) ctx->err = msg; else g_create_error = msg;
  return st;
}

mlmc_status mlmc::cuda_fail(mlmc_ctx* ctx, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(ctx, e == cudaErrorMemoryAllocation ? MLMC_ERR_OOM : MLMC_ERR_CUDA, m);
}



// --------------------------------------------------------------- workspace
// FP32 inner solves are used only where c dt max r' <= mixed_cdr_max (default
// 2), max r' = c((1+a)^2/3 - a).  On strongly indefinite levels the
// continuation's FP32 pseudo-steps can end in a different root than FP64
// ones (measured on the 3D 64x64x16 level at c dt max r' = 2.37; not on the
// 2D 32^2 level at the same value, whose workload raises the limit).
bool mlmc::level_mixed(const mlmc_config& c, const LevelDesc& lv) {
  if (c.precision != MLMC_PREC_MIXED) return false;
  double rmax = c.c * ((1.0 + c.a) * (1.0 + c.a) / 3.0 - c.a);
  double lim = c.mixed_cdr_max > 0.0 ? c.mixed_cdr_max : 2.0;
  return lv.dt * rmax <= lim;
}

// Geometric multigrid preconditioner of a level (row a7): requested by
// cfg.precond and used only where every step Hessian is positive definite,
// c dt max r' < 1, so that the Newton-CG directions -- and the selected root --
// do not depend on the preconditioner beyond the CG tolerance.  mg->G = 0 when
// the level keeps Jacobi.
static bool level_gmg(const mlmc_config& c, const LevelDesc& lv, MGDesc* mg) {
  mg->G = 0;
  mg->per_sample = 0;
  if (c.precond != MLMC_PRECOND_GMG || lv.dim < 2) return false;
  double rmax = c.c * ((1.0 + c.a) * (1.0 + c.a) / 3.0 - c.a);
  if (lv.dt * rmax >= 1.0) return false;
  mg_hierarchy(lv, c.mg_nu > 0 ? c.mg_nu : 2, c.mg_coarse_sweeps > 0 ? c.mg_coarse_sweeps : 8, mg);
  return true;
}

SolveWs mlmc::solve_ws(const mlmc_config& c, const LevelDesc& lv, int n, bool mixed) {
  SolveWs w;
  size_t N = (size_t)lv.nodes, NO = (size_t)n_offsets(lv.dim), kr = mixed ? 4 : 8;
  MGDesc mg;
  level_gmg(c, lv, &mg);
  size_t off = 0;
  w.coef64 = off; off += align256((size_t)n * NO * N * 8);
  w.coef32 = off; off += mixed ? align256((size_t)n * NO * N * 4) : 0;
  w.ubuf = off; off += align256((size_t)n * 2 * N * 8);
  w.F = off; off += align256((size_t)n * N * 8);
  w.Ku = off; off += align256((size_t)n * N * 8);
  w.Kd = off; off += align256((size_t)n * N * 8);
  w.kr = off; off += align256((size_t)n * 7 * N * kr);
  w.mg = off; off += align256((size_t)n * (size_t)mg.per_sample * kr);
  // group layout (global-memory levels): tickets, barrier counters, partials
  w.grp = off;
  if (lv.dim == 3)
    off += align256(group_sync_bytes(GROUP_MAX_SAMPLES)) + align256((size_t)16 * GROUP_MAX_GRID * 8);
  w.total = off;
  return w;
}

PairWs mlmc::pair_ws(const mlmc_ctx* c, int level, int n) {
  PairWs w;
  const LevelDesc& lf = c->lv[level];
  size_t off = 0;
  w.xi = off; off += align256((size_t)n * c->M * 8);
  w.kl = off; off += c->cfg.precision == MLMC_PREC_MIXED ? kl_tc_workspace_bytes(c->M, n) : 0;
  w.Zf = off; off += align256((size_t)n * lf.cells * 8);
  w.Zc = off; off += level > 0 ? align256((size_t)n * c->lv[level - 1].cells * 8) : 0;
  w.tf = off; off += align256((size_t)n * lf.nodes * 8);
  w.tc = off; off += level > 0 ? align256((size_t)n * c->lv[level - 1].nodes * 8) : 0;
  w.info = off; off += align256((size_t)2 * n * sizeof(mlmc_sample_info));
  w.solve_f = off; off += solve_ws(c->cfg, lf, n, level_mixed(c->cfg, lf)).total;
  w.solve_c = off;
  if (level > 0) off += solve_ws(c->cfg, c->lv[level - 1], n, level_mixed(c->cfg, c->lv[level - 1])).total;
  w.total = off;
  return w;
}

static bool check_ws(mlmc_ctx* ctx, void* ws, size_t have, size_t need) {
  if (!ws || have < need || ((uintptr_t)ws & 255)) {
    char b[160];
    snprintf(b, sizeof b, "workspace %p of %zu bytes: need %zu bytes, 256-byte aligned", ws, have,
             need);
    ctx->err = b;
    return false;
  }
  return true;
}

// Time scheme, stimulus and QoI fields of a configuration.
bool mlmc::model_config_ok(const mlmc_config& c) {
  if (c.time_scheme != MLMC_SCHEME_IE && c.time_scheme != MLMC_SCHEME_CN) return false;
  if (c.qoi != MLMC_QOI_ACTIVATION && c.qoi != MLMC_QOI_FINAL_STATE) return false;
  if (c.stim_kind == MLMC_STIM_BALL) return true;
  return c.stim_kind == MLMC_STIM_PULSE && c.stim_sigma > 0.0 && c.stim_t1 >= 0.0 &&
         c.stim_amp == c.stim_amp;
}

// Geometry of level `level` of a configuration: n0[d] 2^level cells per axis,
// m0 2^level implicit-Euler steps.  False (and a message) when a size does not
// fit the kernels' index types.
bool mlmc::derive_level(const mlmc_config& c, int level, LevelDesc* out, std::string* err) {
  LevelDesc lv;
  lv.dim = c.dim;
  int64_t nodes = 1, cells = 1;
  double vol = 1.0;
  if (level < 0 || level >= MLMC_MAX_LEVELS) { *err = "level out of range"; return false; }
  for (int d = 0; d < 3; ++d) {
    if (d < c.dim) {
      if (c.n0[d] < 1 || !(c.L[d] > 0.0)) { *err = "n0 and L must be positive"; return false; }
      int64_t nn = (int64_t)c.n0[d] << level;
      if (nn > (1 << 20)) { *err = "grid too large"; return false; }
      lv.n[d] = (int)nn; lv.N[d] = (int)nn + 1; lv.h[d] = c.L[d] / (double)nn;
    } else {
      lv.n[d] = 1; lv.N[d] = 1; lv.h[d] = 1.0;
    }
    nodes *= lv.N[d]; cells *= lv.n[d]; vol *= (d < c.dim ? lv.h[d] : 1.0);
  }
  if (nodes > (int64_t)1 << 31) { *err = "grid too large"; return false; }
  const int64_t m = (int64_t)c.m0 << level;
  if (c.m0 < 1 || m > (int64_t)1 << 30) { *err = "time steps out of range"; return false; }
  lv.nodes = nodes; lv.cells = cells; lv.vol = vol;
  lv.m = (int)m;
  lv.T = c.T;
  lv.dt = c.T / (double)lv.m;
  *out = lv;
  return true;
}

void mlmc::derive_physics(const mlmc_config& c, Physics* out) {
  const double pi = 3.141592653589793238462643;
  Physics ph;
  ph.stim_ps = nullptr;
  ph.c = c.c; ph.a = c.a; ph.s_t = c.s_t; ph.s_l0 = c.s_l0;
  ph.th0 = c.theta0_deg * pi / 180.0;
  ph.th1 = c.theta1_deg * pi / 180.0;
  ph.Lz = c.dim == 3 ? c.L[2] : 1.0;
  ph.stim_r2 = c.stim_r * c.stim_r;
  for (int d = 0; d < 3; ++d) ph.stim_c[d] = c.stim_c[d];
  ph.theta = c.time_scheme == MLMC_SCHEME_CN ? 0.5 : 1.0;
  ph.stim_kind = c.stim_kind;
  ph.stim_amp = c.stim_amp;
  ph.stim_isig2 = c.stim_kind == MLMC_STIM_PULSE ? 1.0 / (c.stim_sigma * c.stim_sigma) : 0.0;
  ph.stim_t1 = c.stim_t1;
  ph.qoi = c.qoi;
  ph.cond_kind = c.kl_kind == MLMC_KL_AFFINE_GAUSSIAN ? 1 : 0;
  *out = ph;
}

// Solver parameters of one level: the configured tolerances (the FP32 inner
// solves no tighter than 1e-5), the root-selection regime of the level
// (gradient-flow continuation where a step has several roots) and the FP32
// range scaling of the fine 3D levels.
SolverParams mlmc::level_solver_params(const mlmc_config& c, const LevelDesc& lv, bool mixed) {
  SolverParams sp;
  sp.newton_tol = c.newton_tol;
  sp.newton_max = c.newton_max;
  sp.lin_rtol = mixed ? fmax(c.lin_rtol, 1e-5) : c.lin_rtol;
  sp.lin_max = c.lin_max;
  sp.ls_full_step = 1e-6;
  sp.flow = level_has_several_roots(c.c, c.a, lv.dt) ? 1 : 0;
  sp.tau0 = 0.5 / (c.c * ((1.0 + c.a) * (1.0 + c.a) / 3.0 - c.a));
  sp.cg_scale = mixed && cg_needs_scaling(lv) ? 1 : 0;
  // the predicated stencil pays where boundary nodes are many (measured: 3D
  // 64x64x16, 17 % boundary nodes, 32.1 -> 24.6 s; the 2D levels) and costs
  // where they are few (3D 128x128x32 and 256x256x64, 8.9 % and 4.6 %: 2.13 ->
  // 2.62 s and 7.05 -> 10.05 s): 3D grids take it above 12 % boundary nodes
  double interior = 1.0;
  for (int d = 0; d < lv.dim; ++d) interior *= (double)(lv.N[d] - 2) / lv.N[d];
  sp.pred_stencil = lv.dim < 3 || 1.0 - interior > 0.12 ? 1 : 0;
  return sp;
}

// --------------------------------------------------------------- create
extern "C" mlmc_status mlmc_create(const mlmc_config* cfg, mlmc_ctx** out) {
  if (!out) return fail(nullptr, MLMC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, MLMC_ERR_ARG, "cfg is NULL");
  const mlmc_config& c = *cfg;
  if (c.dim < 1 || c.dim > 3) return fail(nullptr, MLMC_ERR_ARG, "dim must be 1, 2 or 3");
  if (c.n_levels < 1 || c.n_levels > MLMC_MAX_LEVELS)
    return fail(nullptr, MLMC_ERR_ARG, "n_levels out of range");
  for (int d = 0; d < c.dim; ++d)
    if (c.n0[d] < 1 || !(c.L[d] > 0.0)) return fail(nullptr, MLMC_ERR_ARG, "n0 and L must be positive");
  if (c.m0 < 1 || !(c.T > 0.0)) return fail(nullptr, MLMC_ERR_ARG, "m0 and T must be positive");
  if (c.kl_modes < 1 || c.kl_modes > 4096 || !(c.kl_ell > 0.0) || !(c.kl_sigma2 >= 0.0))
    return fail(nullptr, MLMC_ERR_ARG, "KL parameters out of range");
  if (c.precision != MLMC_PREC_FP64 && c.precision != MLMC_PREC_MIXED)
    return fail(nullptr, MLMC_ERR_ARG, "unknown precision");
  if (!(c.newton_tol > 0.0) || c.newton_max < 1 || !(c.lin_rtol > 0.0) || c.lin_max < 1)
    return fail(nullptr, MLMC_ERR_ARG, "solver tolerances / iteration caps must be positive");
  if (!(c.s_t > 0.0) || !(c.s_l0 > 0.0)) return fail(nullptr, MLMC_ERR_ARG, "conductivities must be positive");
  if (c.solver < MLMC_SOLVER_AUTO || c.solver > MLMC_SOLVER_CLUSTER)
    return fail(nullptr, MLMC_ERR_ARG, "unknown solver layout");
  if (c.cluster_size != 0 && c.cluster_size != 1 && c.cluster_size != 2 && c.cluster_size != 4 &&
      c.cluster_size != 8 && c.cluster_size != 16)
    return fail(nullptr, MLMC_ERR_ARG, "cluster_size must be 0, 1, 2, 4, 8 or 16");
  if (c.precond != MLMC_PRECOND_JACOBI && c.precond != MLMC_PRECOND_GMG)
    return fail(nullptr, MLMC_ERR_ARG, "unknown preconditioner");
  if (c.mg_nu < 0 || c.mg_nu > 8 || c.mg_coarse_sweeps < 0 || c.mg_coarse_sweeps > 64)
    return fail(nullptr, MLMC_ERR_ARG, "mg_nu must be 0..8 and mg_coarse_sweeps 0..64");
  if (!model_config_ok(c)) return fail(nullptr, MLMC_ERR_ARG, "time scheme, stimulus or QoI out of range");
  if (c.kl_kind != MLMC_KL_SEPARABLE_EXP && c.kl_kind != MLMC_KL_AFFINE_GAUSSIAN)
    return fail(nullptr, MLMC_ERR_ARG, "unknown KL kind");
  if (c.kl_kind == MLMC_KL_AFFINE_GAUSSIAN) {
    if (!(c.kl_tol >= 0.0) || !(c.kl_s >= 0.0) || !(c.kl_delta > 0.0 && c.kl_delta < 1.0))
      return fail(nullptr, MLMC_ERR_ARG, "affine KL parameters out of range");
    int64_t cand = 1;
    for (int d = 0; d < c.dim; ++d) {
      if (c.kl_cand_n[d] < 0 || c.kl_cand_n[d] > (1 << 20))
        return fail(nullptr, MLMC_ERR_ARG, "affine KL candidate grid out of range");
      cand *= c.kl_cand_n[d] ? c.kl_cand_n[d] : c.n0[d];
    }
    if (cand > (int64_t)1 << 22) return fail(nullptr, MLMC_ERR_ARG, "affine KL candidate grid too large");
  }

  mlmc_ctx* ctx = new mlmc_ctx();
  ctx->cfg = c;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e != cudaSuccess) { delete ctx; return fail(nullptr, MLMC_ERR_CUDA, cudaGetErrorString(e)); }
  for (int l = 0; l < c.n_levels; ++l) {
    std::string why;
    if (!derive_level(c, l, &ctx->lv[l], &why)) { delete ctx; return fail(nullptr, MLMC_ERR_ARG, why); }
  }
  derive_physics(c, &ctx->ph);
  SolverParams& sp = ctx->sp;
  sp = level_solver_params(c, ctx->lv[0], c.precision == MLMC_PREC_MIXED);   // per level in solve_into

  // KL mode table and per-level 1D mode values at the cell centroids
  ctx->M = c.kl_modes;
  std::vector<int> idx;
  std::vector<double> sl;
  const bool affine = c.kl_kind == MLMC_KL_AFFINE_GAUSSIAN;
  if (affine) {
    idx.assign(3 * c.kl_modes, 0);       // unused: the modes come from the factor
    sl.assign(c.kl_modes, 0.0);          // filled with s_eff below
  } else if (!kl_table_host(c.dim, c.L, c.kl_sigma2, c.kl_ell, c.kl_modes, idx, sl)) {
    delete ctx;
    return fail(nullptr, MLMC_ERR_ARG, "KL mode table could not be built");
  }
  int n1d[3] = {0, 0, 0};
  for (int q = 0; q < c.kl_modes; ++q)
    for (int d = 0; d < 3; ++d) n1d[d] = idx[3 * q + d] + 1 > n1d[d] ? idx[3 * q + d] + 1 : n1d[d];
  auto cleanup_fail = [&](cudaError_t err, const char* where) {
    mlmc_destroy(ctx);
    return fail(nullptr, err == cudaErrorMemoryAllocation ? MLMC_ERR_OOM : MLMC_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(err));
  };
  if ((e = cudaMalloc(&ctx->d_sqrt_lam, sizeof(double) * c.kl_modes)) != cudaSuccess) return cleanup_fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&ctx->d_idx, sizeof(int) * 3 * c.kl_modes)) != cudaSuccess) return cleanup_fail(e, "cudaMalloc");
  if (affine) {
    // the paper's KL: pivoted Cholesky on the candidate grid's centroids,
    // the mode tables of every level, s_eff = min(s, delta / max sum |l_k|)
    // with the max over the candidates
    int cand_n[3] = {1, 1, 1};
    for (int d = 0; d < c.dim; ++d) cand_n[d] = c.kl_cand_n[d] ? c.kl_cand_n[d] : c.n0[d];
    std::vector<double> xp, lpiv;
    double bound = 0.0;
    ctx->kl_rank = pivoted_cholesky_host(c.dim, c.L, cand_n, c.kl_sigma2, c.kl_ell, c.kl_modes,
                                         c.kl_tol, xp, lpiv, &bound);
    if (ctx->kl_rank < 1) { mlmc_destroy(ctx); return fail(nullptr, MLMC_ERR_ARG, "KL factor has rank 0"); }
    if ((e = cudaMalloc(&ctx->d_xp, sizeof(double) * xp.size())) != cudaSuccess) return cleanup_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&ctx->d_lpiv, sizeof(double) * lpiv.size())) != cudaSuccess) return cleanup_fail(e, "cudaMalloc");
    if ((e = cudaMemcpy(ctx->d_xp, xp.data(), sizeof(double) * xp.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e, "cudaMemcpy");
    if ((e = cudaMemcpy(ctx->d_lpiv, lpiv.data(), sizeof(double) * lpiv.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e, "cudaMemcpy");
    for (int l = 0; l < c.n_levels; ++l) {
      const size_t cnt = (size_t)ctx->lv[l].cells * c.kl_modes;
      if ((e = cudaMalloc(&ctx->d_tab64[l], sizeof(double) * cnt)) != cudaSuccess) return cleanup_fail(e, "cudaMalloc");
      if ((e = cudaMalloc(&ctx->d_tab32[l], sizeof(float) * cnt)) != cudaSuccess) return cleanup_fail(e, "cudaMalloc");
      if ((e = launch_pc_eval(ctx->lv[l], c.kl_modes, ctx->kl_rank, c.kl_sigma2, c.kl_ell, ctx->d_xp,
                              ctx->d_lpiv, ctx->d_tab64[l], ctx->d_tab32[l], nullptr, nullptr)) != cudaSuccess)
        return cleanup_fail(e, "pc_eval");
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cleanup_fail(e, "pc_eval");
    ctx->kl_s_eff = bound > 0.0 ? fmin(c.kl_s, c.kl_delta / bound) : c.kl_s;
    for (int q = 0; q < c.kl_modes; ++q) sl[q] = ctx->kl_s_eff;
  }
  if ((e = cudaMemcpy(ctx->d_sqrt_lam, sl.data(), sizeof(double) * c.kl_modes, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e, "cudaMemcpy");
  if ((e = cudaMemcpy(ctx->d_idx, idx.data(), sizeof(int) * 3 * c.kl_modes, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e, "cudaMemcpy");
  for (int l = 0; l < c.n_levels && !affine; ++l)
    for (int d = 0; d < c.dim; ++d) {
      std::vector<double> tab;
      kl_phi_table_host(c.L[d], c.kl_ell, n1d[d], ctx->lv[l].n[d], tab);
      if ((e = cudaMalloc(&ctx->d_phi[l][d], sizeof(double) * tab.size())) != cudaSuccess) return cleanup_fail(e, "cudaMalloc");
      if ((e = cudaMemcpy(ctx->d_phi[l][d], tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e, "cudaMemcpy");
      std::vector<float> tab32(tab.begin(), tab.end());
      if ((e = cudaMalloc(&ctx->d_phi32[l][d], sizeof(float) * tab32.size())) != cudaSuccess) return cleanup_fail(e, "cudaMalloc");
      if ((e = cudaMemcpy(ctx->d_phi32[l][d], tab32.data(), sizeof(float) * tab32.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e, "cudaMemcpy");
    }
  int64_t n0 = ctx->lv[0].nodes;
  int L = c.n_levels;
  size_t est = (size_t)(2 * n0 + 2 * (int64_t)L * n0 + L + 2);
  if ((e = cudaMalloc(&ctx->d_acc, sizeof(double) * 3 * L * n0)) != cudaSuccess) return cleanup_fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&ctx->d_N, sizeof(int64_t) * L)) != cudaSuccess) return cleanup_fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&ctx->d_est, sizeof(double) * est)) != cudaSuccess) return cleanup_fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&ctx->d_cnt, sizeof(unsigned long long) * N_COUNTERS)) != cudaSuccess) return cleanup_fail(e, "cudaMalloc");
  if ((e = cudaMemset(ctx->d_acc, 0, sizeof(double) * 3 * L * n0)) != cudaSuccess) return cleanup_fail(e, "cudaMemset");
  if ((e = cudaMemset(ctx->d_cnt, 0, sizeof(unsigned long long) * N_COUNTERS)) != cudaSuccess) return cleanup_fail(e, "cudaMemset");
  for (int i = 0; i < 2 * L; ++i)
    if ((e = cudaStreamCreateWithFlags(&ctx->lvl_stream[i], cudaStreamNonBlocking)) != cudaSuccess)
      return cleanup_fail(e, "cudaStreamCreate");
  if ((e = cudaStreamCreateWithFlags(&ctx->aux_pub, cudaStreamNonBlocking)) != cudaSuccess)
    return cleanup_fail(e, "cudaStreamCreate");
  if ((e = preload_kl_tc()) != cudaSuccess) return cleanup_fail(e, "cudaFuncSetAttribute");
  *out = ctx;
  return MLMC_OK;
}

extern "C" void mlmc_destroy(mlmc_ctx* ctx) {
  if (!ctx) return;
  cudaFree(ctx->d_sqrt_lam);
  cudaFree(ctx->d_idx);
  for (int l = 0; l < MLMC_MAX_LEVELS; ++l)
    for (int d = 0; d < 3; ++d) {
      cudaFree(ctx->d_phi[l][d]);
      cudaFree(ctx->d_phi32[l][d]);
    }
  for (int l = 0; l < MLMC_MAX_LEVELS; ++l) {
    cudaFree(ctx->d_tab64[l]);
    cudaFree(ctx->d_tab32[l]);
  }
  cudaFree(ctx->d_xp);
  cudaFree(ctx->d_lpiv);
  cudaFree(ctx->d_acc);
  cudaFree(ctx->d_N);
  cudaFree(ctx->d_est);
  cudaFree(ctx->d_cnt);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->grp_ev) cudaEventDestroy(ctx->grp_ev);
  for (cudaEvent_t ev : ctx->ev_pool) cudaEventDestroy(ev);
  for (cudaEvent_t ev : ctx->sync_pool) cudaEventDestroy(ev);
  for (int i = 0; i < 2 * MLMC_MAX_LEVELS; ++i)
    if (ctx->lvl_stream[i]) cudaStreamDestroy(ctx->lvl_stream[i]);
  if (ctx->aux_pub) cudaStreamDestroy(ctx->aux_pub);
  delete ctx;
}

extern "C" const char* mlmc_last_error(const mlmc_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

// Make `waiter` wait for the work enqueued so far on `src` (an ordering-only
// event from the context's pool).
mlmc_status mlmc::order_after(mlmc_ctx* ctx, cudaStream_t src, cudaStream_t waiter) {
  if (src == waiter) return MLMC_OK;
  if (ctx->sync_used == ctx->sync_pool.size()) {
    cudaEvent_t ev;
    CK(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    ctx->sync_pool.push_back(ev);
  }
  cudaEvent_t ev = ctx->sync_pool[ctx->sync_used++];
  CK(ctx, cudaEventRecord(ev, src));
  CK(ctx, cudaStreamWaitEvent(waiter, ev, 0));
  return MLMC_OK;
}

static bool bad_level(mlmc_ctx* ctx, int level) {
  if (level < 0 || level >= ctx->cfg.n_levels) {
    ctx->err = "level out of range";
    return true;
  }
  return false;
}

extern "C" mlmc_status mlmc_level_info(const mlmc_ctx* ctx, int level, int64_t* nodes,
                                       int64_t* cells, int32_t* steps) {
  if (!ctx) return MLMC_ERR_ARG;
  if (level < 0 || level >= ctx->cfg.n_levels) return MLMC_ERR_ARG;
  if (nodes) *nodes = ctx->lv[level].nodes;
  if (cells) *cells = ctx->lv[level].cells;
  if (steps) *steps = ctx->lv[level].m;
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_workspace_bytes(const mlmc_ctx* ctx, int level, int n, size_t* bytes) {
  if (!ctx || !bytes || n < 0) return MLMC_ERR_ARG;
  if (level < 0 || level >= ctx->cfg.n_levels) return MLMC_ERR_ARG;
  *bytes = pair_ws(ctx, level, n).total;
  return MLMC_OK;
}

// --------------------------------------------------------------- steps
extern "C" mlmc_status mlmc_xi(mlmc_ctx* ctx, uint64_t seed, int level, const uint64_t* ids, int n,
                               double* xi, void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  if (n < 0 || (n > 0 && (!ids || !xi))) return fail(ctx, MLMC_ERR_ARG, "mlmc_xi: bad arguments");
  if (level < 0) return fail(ctx, MLMC_ERR_ARG, "mlmc_xi: negative level");
  CK(ctx, launch_xi(seed, nullptr, level, ids, n, ctx->M, ctx->cfg.kl_kind, xi, (cudaStream_t)stream));
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_kl_field(mlmc_ctx* ctx, int level, const double* xi, int n, double* Z,
                                     void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  if (bad_level(ctx, level)) return MLMC_ERR_ARG;
  if (n < 0 || (n > 0 && (!xi || !Z))) return fail(ctx, MLMC_ERR_ARG, "mlmc_kl_field: bad arguments");
  if (ctx->cfg.kl_kind == MLMC_KL_AFFINE_GAUSSIAN)
    CK(ctx, launch_kl_field_table(ctx->lv[level], ctx->M, ctx->d_sqrt_lam, ctx->d_tab64[level], xi, n,
                                  Z, (cudaStream_t)stream));
  else
    CK(ctx, launch_kl_field(ctx->lv[level], ctx->M, ctx->d_sqrt_lam, ctx->d_idx, ctx->d_phi[level][0],
                            ctx->d_phi[level][1], ctx->d_phi[level][2], 0, xi, n, Z,
                            (cudaStream_t)stream));
  ctx->launches += 1;
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_kl_tc_workspace_bytes(const mlmc_ctx* ctx, int n, size_t* bytes) {
  if (!ctx || !bytes || n < 0) return MLMC_ERR_ARG;
  *bytes = kl_tc_workspace_bytes(ctx->M, n);
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_kl_field_tc(mlmc_ctx* ctx, int level, const double* xi, int n,
                                        double* Z, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  if (bad_level(ctx, level)) return MLMC_ERR_ARG;
  if (n < 0 || n > 65535 * 256 || (n > 0 && (!xi || !Z)))
    return fail(ctx, MLMC_ERR_ARG, "mlmc_kl_field_tc: bad arguments");
  if (n == 0) return MLMC_OK;
  if (!check_ws(ctx, ws, ws_bytes, kl_tc_workspace_bytes(ctx->M, n))) return MLMC_ERR_WORKSPACE;
  CK(ctx, launch_kl_field_tc(ctx->lv[level], ctx->M, ctx->d_sqrt_lam, ctx->d_idx,
                             ctx->d_phi32[level][0], ctx->d_phi32[level][1],
                             ctx->d_phi32[level][2], ctx->d_tab32[level], xi, n, Z, ws,
                             ctx->d_cnt + CNT_TC_TIMEOUT,
                             ctx->tc_check_limit, (cudaStream_t)stream));
  ctx->launches += 2;
  return MLMC_OK;
}

// The KL field of the pipeline: on the tensor cores (split TF32) on levels
// whose inner solves run in FP32 (MLMC_PREC_MIXED and c dt max r' <=
// mixed_cdr_max) and whose steps are at most mildly indefinite (c dt max r'
// <= 2), in FP64 elsewhere -- where the root selection is sensitive to
// perturbations of the field, the field stays exact to FP64 rounding.
// kws: kl_tc_workspace_bytes(M, n) bytes of the pair workspace.
static mlmc_status kl_into(mlmc_ctx* ctx, int level, const double* xi, int n, double* Z,
                           char* kws, cudaStream_t st) {
  const mlmc_config& c = ctx->cfg;
  const double cdr = ctx->lv[level].dt * c.c * ((1.0 + c.a) * (1.0 + c.a) / 3.0 - c.a);
  if (level_mixed(c, ctx->lv[level]) && cdr <= 2.0)
    return mlmc_kl_field_tc(ctx, level, xi, n, Z, kws, kl_tc_workspace_bytes(ctx->M, n), st);
  return mlmc_kl_field(ctx, level, xi, n, Z, st);
}

// Coefficients + sweep for n samples of one level inside an already checked
// workspace region.
// The solve layout of a level for a launch of n samples: false = the
// block-per-sample kernel, else a cluster or group plan.  Layout codes
// (mlmc_set_layout): -1 block kernel, 0 automatic (the smallest shared-memory
// cluster that holds a sample; else, on 3D grids, the group layout when it
// gives a sample at least 32 CTAs; else global-memory clusters of 16), 1..16
// shared-memory clusters of that size, 100 + C global-memory clusters of C
// CTAs (300 + C: of 256-thread CTAs), MLMC_LAYOUT_GROUP the group layout.
static bool choose_plan(const mlmc_ctx* ctx, const LevelDesc& lv, bool mixed, int level, int n,
                        ClusterPlan* plan) {
  if (ctx->cfg.solver == MLMC_SOLVER_BLOCK) return false;
  const int want = ctx->cfg.cluster_size ? ctx->cfg.cluster_size : ctx->tuned_C[level];
  if (want < 0 && ctx->cfg.solver == MLMC_SOLVER_AUTO) return false;
  bool ok = false;
  MGDesc mg;
  const bool gmg = level_gmg(ctx->cfg, lv, &mg);
  if (want == MLMC_LAYOUT_GROUP) {   // (multigrid levels keep clusters)
    if (!gmg && group_plan(lv, mixed, n, true, plan, &ok) == cudaSuccess && ok) return true;
    return cluster_plan(lv, mixed, 0, plan, true);
  }
  if (want > 300) return cluster_plan(lv, mixed, want - 300, plan, true, 256);
  if (want > 100) return cluster_plan(lv, mixed, want - 100, plan, true);
  if (want > 0 && cluster_plan(lv, mixed, want, plan)) return true;
  if (want == 0 && gmg) return cluster_plan(lv, mixed, 0, plan, true);
  if (cluster_plan(lv, mixed, 0, plan)) return true;
  if (want == 0 && group_plan(lv, mixed, n, false, plan, &ok) == cudaSuccess && ok) return true;
  return cluster_plan(lv, mixed, 0, plan, true);
}

static bool valid_layout(int C) {
  const int ok[18] = {-1, 0, 1, 2, 4, 8, 16, 101, 102, 104, 108, 116,
                      301, 302, 304, 308, 316, MLMC_LAYOUT_GROUP};
  for (int v : ok)
    if (C == v) return true;
  return false;
}

static mlmc_status solve_into(mlmc_ctx* ctx, int level, const double* Z, int n, double* t_act,
                              double* slab, mlmc_sample_info* info, char* ws, cudaStream_t st,
                              const double* stim = nullptr) {
  Physics ph = ctx->ph;
  ph.stim_ps = stim;
  const LevelDesc& lv = ctx->lv[level];
  bool mixed = level_mixed(ctx->cfg, lv);
  SolveWs w = solve_ws(ctx->cfg, lv, n, mixed);
  double* coef64 = (double*)(ws + w.coef64);
  float* coef32 = mixed ? (float*)(ws + w.coef32) : nullptr;
  ClusterPlan plan;
  const bool use_cluster = choose_plan(ctx, lv, mixed, level, n, &plan);
  if (ctx->cfg.solver == MLMC_SOLVER_CLUSTER && !use_cluster)
    return fail(ctx, MLMC_ERR_ARG, "cluster layout requested but no cluster plan fits");
  MGDesc mg;
  level_gmg(ctx->cfg, lv, &mg);
  // the 3D global-memory sweeps (clusters and groups, Jacobi) read each
  // symmetric coupling pair stored once
  const bool sym = use_cluster && plan.gm && lv.dim == 3 && mg.G == 0;
  CK(ctx, launch_assemble(lv, ph, Z, n, coef64, coef32, st, sym));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ctx->prof) {
    while (ctx->ev_pool.size() < ctx->ev_used + 2) {
      cudaEvent_t ev;
      CK(ctx, cudaEventCreate(&ev));
      ctx->ev_pool.push_back(ev);
    }
    e0 = ctx->ev_pool[ctx->ev_used++];
    e1 = ctx->ev_pool[ctx->ev_used++];
    ctx->ev_level.push_back(ctx->prof_level);
    ctx->ev_grid.push_back(level);
    CK(ctx, cudaEventRecordWithFlags(e0, st, ctx->capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
  }
  SolverParams sp = level_solver_params(ctx->cfg, lv, mixed);
  sp.grp_check = ctx->tc_check_limit;
  if (use_cluster) {
    ClusterGlobal g;
    g.u = (double*)(ws + w.ubuf);
    g.F = (double*)(ws + w.F);
    g.kr = (void*)(ws + w.kr);
    g.code = (unsigned*)(ws + w.Ku);
    g.mg = mg.G > 0 ? (void*)(ws + w.mg) : nullptr;
    if (plan.G > 0) {
      g.gsync = (unsigned*)(ws + w.grp);
      g.gslot = (double*)(ws + w.grp + align256(group_sync_bytes(GROUP_MAX_SAMPLES)));
      // group launches of this context run one after another
      if (ctx->grp_ev_valid) CK(ctx, cudaStreamWaitEvent(st, ctx->grp_ev, 0));
    }
    CK(ctx, launch_solve_cluster(lv, ph, sp, mixed, plan, n, coef64, coef32, slab, t_act, info,
                                 ctx->d_cnt + CNT_LEVEL + CNT_PER_LEVEL * level, g, mg, st));
    if (plan.G > 0) {
      if (!ctx->grp_ev) CK(ctx, cudaEventCreateWithFlags(&ctx->grp_ev, cudaEventDisableTiming));
      CK(ctx, cudaEventRecord(ctx->grp_ev, st));
      ctx->grp_ev_valid = true;
    }
  }
  else
    CK(ctx, launch_solve(lv, ph, sp, mixed, n, coef64, coef32, slab, (double*)(ws + w.ubuf),
                         (double*)(ws + w.F), (double*)(ws + w.Ku), (double*)(ws + w.Kd),
                         (void*)(ws + w.kr), t_act, info,
                         ctx->d_cnt + CNT_LEVEL + CNT_PER_LEVEL * level, st));
  if (ctx->prof)
    CK(ctx, cudaEventRecordWithFlags(e1, st, ctx->capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
  ctx->launches += 2;
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_solve(mlmc_ctx* ctx, int level, const double* Z, int n, double* t_act,
                                  double* slab, mlmc_sample_info* info, void* ws, size_t ws_bytes,
                                  void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  if (bad_level(ctx, level)) return MLMC_ERR_ARG;
  if (n < 0 || n > 65535 || (n > 0 && (!Z || !t_act)))
    return fail(ctx, MLMC_ERR_ARG, "mlmc_solve: bad arguments");
  size_t need = solve_ws(ctx->cfg, ctx->lv[level], n, level_mixed(ctx->cfg, ctx->lv[level])).total;
  if (!check_ws(ctx, ws, ws_bytes, need)) return MLMC_ERR_WORKSPACE;
  if (n == 0) return MLMC_OK;
  return solve_into(ctx, level, Z, n, t_act, slab, info, (char*)ws, (cudaStream_t)stream);
}

// Autotuner: the solve kernel's layout for one level (block-per-sample, or a
// cluster of C = 1..16 CTAs per sample, each with its own band height) is
// timed on n samples of the level with CUDA events and the fastest is kept.
extern "C" mlmc_status mlmc_autotune(mlmc_ctx* ctx, int level, uint64_t seed, const uint64_t* ids,
                                     int n, void* ws, size_t ws_bytes, int* best, float* ms,
                                     void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  if (bad_level(ctx, level)) return MLMC_ERR_ARG;
  if (n < 1 || n > 65535 || !ids) return fail(ctx, MLMC_ERR_ARG, "mlmc_autotune: bad arguments");
  if (!check_ws(ctx, ws, ws_bytes, pair_ws(ctx, level, n).total)) return MLMC_ERR_WORKSPACE;
  const LevelDesc& lv = ctx->lv[level];
  const bool mixed = level_mixed(ctx->cfg, lv);
  cudaStream_t st = (cudaStream_t)stream;
  PairWs w = pair_ws(ctx, level, n);
  char* p = (char*)ws;
  double* xi = (double*)(p + w.xi);
  double* Z = (double*)(p + w.Zf);
  double* t = (double*)(p + w.tf);
  mlmc_sample_info* inf = (mlmc_sample_info*)(p + w.info);
  CK(ctx, launch_xi(seed, nullptr, level, ids, n, ctx->M, ctx->cfg.kl_kind, xi, st));
  mlmc_status r;
  if ((r = mlmc_kl_field(ctx, level, xi, n, Z, st)) != MLMC_OK) return r;
  // candidates: the block kernel (only when the layout is not forced), shared-
  // memory clusters of 1..16 CTAs (where a band fits), global-memory clusters
  const int cand[MLMC_TUNE_CANDIDATES] = {-1, 1, 2, 4, 8, 16, 101, 102, 104, 108, 116,
                                          301, 302, 304, 308, MLMC_LAYOUT_GROUP};
  float t_ms[MLMC_TUNE_CANDIDATES];
  int choice = 0;
  float best_ms = 0.f;
  const int saved = ctx->tuned_C[level];
  const bool saved_prof = ctx->prof;
  ctx->prof = false;
  struct Restore {
    mlmc_ctx* c; int l; int v; bool pr;
    ~Restore() { c->tuned_C[l] = v; c->prof = pr; }
  } restore{ctx, level, saved, saved_prof};
  cudaEvent_t e[2];
  CK(ctx, cudaEventCreate(&e[0]));
  CK(ctx, cudaEventCreate(&e[1]));
  struct EvFree { cudaEvent_t* e; ~EvFree() { cudaEventDestroy(e[0]); cudaEventDestroy(e[1]); } } ev_free{e};
  for (int i = 0; i < MLMC_TUNE_CANDIDATES; ++i) {
    t_ms[i] = -1.f;
    const int C = cand[i];
    if (C < 0 && ctx->cfg.solver != MLMC_SOLVER_AUTO) continue;
    if (C > 0) {
      ClusterPlan pl;
      if (ctx->cfg.solver == MLMC_SOLVER_BLOCK) continue;
      if (C == MLMC_LAYOUT_GROUP) {
        bool gok = false;
        CK(ctx, group_plan(lv, mixed, n, true, &pl, &gok));
        if (!gok) continue;
      } else if (!cluster_plan(lv, mixed, C > 300 ? C - 300 : (C > 100 ? C - 100 : C), &pl, C > 100,
                               C > 300 ? 256 : 512)) {
        continue;
      }
      int active = 0;
      CK(ctx, cluster_max_active(lv, mixed, pl, &active));
      if (active < 1) continue;
    } else {
      CK(ctx, preload_solve(lv, mixed));
    }
    ctx->tuned_C[level] = C;
    const int force = ctx->cfg.cluster_size;
    ctx->cfg.cluster_size = 0;
    CK(ctx, cudaEventRecord(e[0], st));
    r = solve_into(ctx, level, Z, n, t, nullptr, inf, p + w.solve_f, st);
    ctx->cfg.cluster_size = force;
    if (r != MLMC_OK) return r;
    CK(ctx, cudaEventRecord(e[1], st));
    CK(ctx, cudaEventSynchronize(e[1]));
    CK(ctx, cudaEventElapsedTime(&t_ms[i], e[0], e[1]));
    if (best_ms == 0.f || t_ms[i] < best_ms) { best_ms = t_ms[i]; choice = C; }
  }
  if (best_ms == 0.f) return fail(ctx, MLMC_ERR_ARG, "mlmc_autotune: no solver layout fits this level");
  restore.v = choice;
  if (best) *best = choice;
  if (ms) memcpy(ms, t_ms, sizeof t_ms);
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_get_layout(const mlmc_ctx* ctx, int level, int* C) {
  if (!ctx || !C || level < 0 || level >= ctx->cfg.n_levels) return MLMC_ERR_ARG;
  *C = ctx->cfg.cluster_size ? ctx->cfg.cluster_size : ctx->tuned_C[level];
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_set_layout(mlmc_ctx* ctx, int level, int C) {
  if (!ctx) return MLMC_ERR_ARG;
  if (bad_level(ctx, level) || !valid_layout(C))
    return fail(ctx, MLMC_ERR_ARG, "mlmc_set_layout: level or layout out of range");
  ctx->tuned_C[level] = C;
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_slab_residual(mlmc_ctx* ctx, int level, const double* Z,
                                          const double* slab, int n, double* F, double* res_max,
                                          void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  if (bad_level(ctx, level)) return MLMC_ERR_ARG;
  if (n < 0 || n > 65535 || (n > 0 && (!Z || !slab)))
    return fail(ctx, MLMC_ERR_ARG, "mlmc_slab_residual: bad arguments");
  if (n == 0) return MLMC_OK;
  const LevelDesc& lv = ctx->lv[level];
  // couplings are rebuilt into a context-independent scratch owned by this call
  double* coef = nullptr;
  size_t bytes = (size_t)n * n_offsets(lv.dim) * lv.nodes * 8;
  cudaStream_t st = (cudaStream_t)stream;
  CK(ctx, cudaMallocAsync((void**)&coef, bytes, st));
  cudaError_t e = launch_assemble(lv, ctx->ph, Z, n, coef, nullptr, st);
  if (e == cudaSuccess) e = launch_slab_residual(lv, ctx->ph, coef, slab, n, F, res_max, st);
  cudaError_t e2 = cudaFreeAsync(coef, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "mlmc_slab_residual");
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaFreeAsync");
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_activation(mlmc_ctx* ctx, int level, const double* slab, int n,
                                       double* t_act, void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  if (bad_level(ctx, level)) return MLMC_ERR_ARG;
  if (n < 0 || (n > 0 && (!slab || !t_act))) return fail(ctx, MLMC_ERR_ARG, "mlmc_activation: bad arguments");
  CK(ctx, launch_activation(ctx->lv[level], slab, n, t_act, (cudaStream_t)stream));
  return MLMC_OK;
}

// One batch of level-l pairs: xi and both fields on st_f, the fine solve on
// st_f and the coarse solve concurrently on st_c, then the differences on st_f.
mlmc_status mlmc::sample_level_into(mlmc_ctx* ctx, int level, uint64_t seed, const uint64_t* seeds,
                                    const uint64_t* ids, const double* stim, int n, double* y,
                                    double* y2, double* t_fine, double* t_coarse,
                                    mlmc_sample_info* info, char* ws, cudaStream_t st_f,
                                    cudaStream_t st_c) {
  PairWs w = pair_ws(ctx, level, n);
  double* xi = (double*)(ws + w.xi);
  double* Zf = (double*)(ws + w.Zf);
  double* tf = t_fine ? t_fine : (double*)(ws + w.tf);
  mlmc_sample_info* inf = info ? info : (mlmc_sample_info*)(ws + w.info);
  CK(ctx, launch_xi(seed, seeds, level, ids, n, ctx->M, ctx->cfg.kl_kind, xi, st_f));
  ctx->launches += 1;
  mlmc_status r;
  if ((r = kl_into(ctx, level, xi, n, Zf, ws + w.kl, st_f)) != MLMC_OK) return r;
  double* tc = nullptr;
  if (level > 0) {
    double* Zc = (double*)(ws + w.Zc);
    tc = t_coarse ? t_coarse : (double*)(ws + w.tc);
    if ((r = kl_into(ctx, level - 1, xi, n, Zc, ws + w.kl, st_f)) != MLMC_OK) return r;
    if ((r = order_after(ctx, st_f, st_c)) != MLMC_OK) return r;
    if ((r = solve_into(ctx, level - 1, Zc, n, tc, nullptr, inf + n, ws + w.solve_c, st_c, stim)) !=
        MLMC_OK)
      return r;
  }
  if ((r = solve_into(ctx, level, Zf, n, tf, nullptr, inf, ws + w.solve_f, st_f, stim)) != MLMC_OK)
    return r;
  if (level > 0 && (r = order_after(ctx, st_c, st_f)) != MLMC_OK) return r;
  CK(ctx, launch_pair_diff(ctx->lv[0], ctx->lv[level], level > 0 ? &ctx->lv[level - 1] : nullptr, tf,
                           tc, n, y, y2, ctx->d_cnt + CNT_CENSORED + level, st_f));
  ctx->launches += 1;
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_sample_level(mlmc_ctx* ctx, int level, uint64_t seed,
                                         const uint64_t* ids, int n, double* y, double* y2,
                                         double* t_fine, double* t_coarse, mlmc_sample_info* info,
                                         void* ws, size_t ws_bytes, void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  if (bad_level(ctx, level)) return MLMC_ERR_ARG;
  if (n < 0 || n > 65535 || (n > 0 && (!ids || !y || !y2)))
    return fail(ctx, MLMC_ERR_ARG, "mlmc_sample_level: bad arguments");
  if (!check_ws(ctx, ws, ws_bytes, pair_ws(ctx, level, n).total)) return MLMC_ERR_WORKSPACE;
  if (n == 0) return MLMC_OK;
  ctx->sync_used = 0;
  return sample_level_into(ctx, level, seed, nullptr, ids, nullptr, n, y, y2, t_fine, t_coarse, info,
                           (char*)ws, (cudaStream_t)stream, ctx->aux_pub);
}

extern "C" mlmc_status mlmc_reset(mlmc_ctx* ctx, void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(ctx, cudaMemsetAsync(ctx->d_acc, 0, sizeof(double) * 3 * ctx->cfg.n_levels * ctx->lv[0].nodes, st));
  CK(ctx, cudaMemsetAsync(ctx->d_cnt, 0, sizeof(unsigned long long) * N_COUNTERS, st));
  for (int l = 0; l < MLMC_MAX_LEVELS; ++l) ctx->N_acc[l] = 0;
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_accumulate(mlmc_ctx* ctx, int level, const double* y, const double* y2,
                                       int n, void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  if (bad_level(ctx, level)) return MLMC_ERR_ARG;
  if (n < 0 || (n > 0 && (!y || !y2))) return fail(ctx, MLMC_ERR_ARG, "mlmc_accumulate: bad arguments");
  int64_t n0 = ctx->lv[0].nodes, L = ctx->cfg.n_levels;
  double* mean = ctx->d_acc + (int64_t)level * n0;
  CK(ctx, launch_accumulate(n0, y, y2, n, ctx->N_acc[level], mean, mean + L * n0, mean + 2 * L * n0,
                            (cudaStream_t)stream));
  ctx->launches += 1;
  ctx->N_acc[level] += n;
  return MLMC_OK;
}

mlmc_status mlmc::estimate_impl(mlmc_ctx* ctx, double* mean, double* var, double* mean_l,
                                double* var_l, double* V_l, int64_t* N_l, double* rmse,
                                double* bias, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int L = ctx->cfg.n_levels;
  int64_t n0 = ctx->lv[0].nodes;
  std::vector<int64_t> Nh(ctx->N_acc, ctx->N_acc + L);
  CK(ctx, cudaMemcpyAsync(ctx->d_N, Nh.data(), sizeof(int64_t) * L, cudaMemcpyHostToDevice, st));
  CK(ctx, launch_estimate(L, n0, ctx->lv[0], ctx->d_N, ctx->d_acc, ctx->d_acc + (int64_t)L * n0,
                          ctx->d_acc + 2 * (int64_t)L * n0, ctx->d_est, st));
  ctx->launches += 1;
  size_t est = (size_t)(2 * n0 + 2 * (int64_t)L * n0 + L + 2);
  std::vector<double> h(est);
  CK(ctx, cudaMemcpyAsync(h.data(), ctx->d_est, sizeof(double) * est, cudaMemcpyDeviceToHost, st));
  CK(ctx, cudaStreamSynchronize(st));
  const double* p = h.data();
  if (mean) memcpy(mean, p, sizeof(double) * n0);
  if (var) memcpy(var, p + n0, sizeof(double) * n0);
  if (mean_l) memcpy(mean_l, p + 2 * n0, sizeof(double) * L * n0);
  if (var_l) memcpy(var_l, p + 2 * n0 + (int64_t)L * n0, sizeof(double) * L * n0);
  const double* Vp = p + 2 * n0 + 2 * (int64_t)L * n0;
  if (V_l) memcpy(V_l, Vp, sizeof(double) * L);
  if (N_l) memcpy(N_l, Nh.data(), sizeof(int64_t) * L);
  if (bias) *bias = Vp[L];
  if (rmse) *rmse = Vp[L + 1];
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_estimate(mlmc_ctx* ctx, double* mean, double* var, double* mean_l,
                                     double* var_l, double* V_l, int64_t* N_l, double* rmse,
                                     void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  return estimate_impl(ctx, mean, var, mean_l, var_l, V_l, N_l, rmse, nullptr, stream);
}

// --------------------------------------------------------------- whole run
// mlmc_run workspace: per level, ids, y, y2 and a pair workspace for
// min(batch, N_l) pairs, so that all levels can run concurrently.
static size_t level_run_ws(const mlmc_ctx* c, int l, int nb) {
  return align256((size_t)nb * 8) + 2 * align256((size_t)nb * c->lv[0].nodes * 8) +
         pair_ws(c, l, nb).total;
}

static int level_batch(int64_t N, int batch) { return (int)(N < batch ? (N > 0 ? N : 1) : batch); }

// Samples per launch of level l's pairs inside mlmc_run: the whole batch,
// except where a grid of the pair is a 3D grid that takes the group layout
// automatically (no shared-memory cluster fits, no multigrid, layout 0 or the
// group layout): there a launch holds at most as many samples as groups of
// >= 32 CTAs fit the device at once.  Larger launches fall back to 16-CTA
// clusters (measured slower: 64 samples of the 64x64x16 level took 354 s as
// one cluster launch against ~34 s per 8 samples in groups); launches of this
// size run one after another.
static int level_cap(const mlmc_ctx* c, int l) {
  int cap = 65535;
  for (int g = l; g >= 0 && g >= l - 1; --g) {
    const LevelDesc& lv = c->lv[g];
    const int want = c->cfg.cluster_size ? c->cfg.cluster_size : c->tuned_C[g];
    if (lv.dim != 3 || (want != 0 && want != MLMC_LAYOUT_GROUP) || c->cfg.solver == MLMC_SOLVER_BLOCK)
      continue;
    const bool mx = level_mixed(c->cfg, lv);
    ClusterPlan pl;
    MGDesc mg;
    if (want == 0 && (cluster_plan(lv, mx, 0, &pl) || level_gmg(c->cfg, lv, &mg))) continue;
    int m = 0;
    if (group_resident_samples(lv, mx, &m) != cudaSuccess) {
      (void)cudaGetLastError();
      continue;
    }
    if (m >= 1 && m < cap) cap = m;
  }
  return cap;
}

static int level_batch(const mlmc_ctx* c, int l, int64_t N, int batch) {
  const int cap = level_cap(c, l);
  return level_batch(N, batch < cap ? batch : cap);
}

static size_t run_ws(const mlmc_ctx* c, const int64_t* N_l, int batch) {
  size_t s = 0;
  for (int l = 0; l < c->cfg.n_levels; ++l) s += level_run_ws(c, l, level_batch(c, l, N_l[l], batch));
  return s;
}

extern "C" mlmc_status mlmc_run_workspace_bytes(const mlmc_ctx* ctx, const int64_t* N_l, int batch,
                                                size_t* bytes) {
  if (!ctx || !bytes || !N_l || batch < 1 || batch > 65535) return MLMC_ERR_ARG;
  for (int l = 0; l < ctx->cfg.n_levels; ++l)
    if (N_l[l] < 0) return MLMC_ERR_ARG;
  *bytes = run_ws(ctx, N_l, batch);
  return MLMC_OK;
}

// Runs count[l] level-l pairs with sample ids first[l] .. first[l]+count[l]-1
// for every level, accumulating into the context's running estimates (no
// reset).  Every level runs on its own pair of context streams, concurrently
// with the others; within a level the fine and coarse solves of a batch run
// concurrently.  Ordered after the work already on st; st waits for it all.
// lvl_ms (host [levels] or NULL) receives each level's summed solve-kernel
// time in ms (the solves of its pairs, fine and coarse).
static mlmc_status enqueue_levels(mlmc_ctx* ctx, const int64_t* first_id, const int64_t* count,
                                  uint64_t seed, int batch, char* ws, cudaStream_t st);

// With cfg.use_graph the schedule of one call is captured from `st` (every
// context stream joins the capture through the fork / join events) and
// launched as one CUDA graph; the executable graph is updated in place when
// the next call has the same topology (other seeds, ids or workspace), else
// instantiated anew.
static mlmc_status run_levels(mlmc_ctx* ctx, const int64_t* first_id, const int64_t* count,
                              uint64_t seed, int batch, char* ws, cudaStream_t st, double* lvl_ms) {
  const int L = ctx->cfg.n_levels;
  mlmc_status r;
  const size_t ev0 = ctx->ev_used;
  const bool graph = ctx->cfg.use_graph != 0 && st != nullptr;
  if (graph) {
    // kernel attributes are set before the capture
    for (int l = 0; l < L; ++l) {
      for (int lv = l; lv >= 0 && lv >= l - 1; --lv) {
        const LevelDesc& d = ctx->lv[lv];
        const bool mx = level_mixed(ctx->cfg, d);
        ClusterPlan pl;
        if (choose_plan(ctx, d, mx, lv, level_batch(ctx, l, count[l], batch), &pl))
          CK(ctx, preload_solve_cluster(d, mx, pl));
        else
          CK(ctx, preload_solve(d, mx));
        bool gok = false;   // any batch size may pick the group layout on 3D grids
        if (d.dim == 3 && group_plan(d, mx, 1, true, &pl, &gok) == cudaSuccess && gok)
          CK(ctx, preload_solve_cluster(d, mx, pl));
      }
    }
    CK(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    ctx->capturing = true;
    ctx->grp_ev_valid = false;   // no waits on events recorded outside the capture
  }
  r = enqueue_levels(ctx, first_id, count, seed, batch, ws, st);
  if (graph) {
    ctx->capturing = false;
    ctx->grp_ev_valid = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (r != MLMC_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    if (ctx->graph_exec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(ctx->graph_exec, g, &info) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
      }
    }
    if (!ctx->graph_exec) {
      e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
      if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        ctx->graph_exec = nullptr;
        return cuda_fail(ctx, e, "cudaGraphInstantiate");
      }
    }
    cudaGraphDestroy(g);
    CK(ctx, cudaGraphLaunch(ctx->graph_exec, st));
    ctx->graph_runs += 1;
  } else if (r != MLMC_OK) {
    return r;
  }
  if (lvl_ms) {
    CK(ctx, cudaStreamSynchronize(st));
    for (int l = 0; l < L; ++l) lvl_ms[l] = 0.0;
    for (size_t i = ev0; i + 1 < ctx->ev_used; i += 2) {
      float ms = 0.f;
      CK(ctx, cudaEventElapsedTime(&ms, ctx->ev_pool[i], ctx->ev_pool[i + 1]));
      lvl_ms[ctx->ev_level[i / 2]] += ms;
    }
  }
  return MLMC_OK;
}

// The launches of run_levels: every level on its own pair of context streams.
static mlmc_status enqueue_levels(mlmc_ctx* ctx, const int64_t* first_id, const int64_t* count,
                                  uint64_t seed, int batch, char* ws, cudaStream_t st) {
  const int L = ctx->cfg.n_levels;
  mlmc_status r;
  ctx->prof = true;
  struct ProfOff { mlmc_ctx* c; ~ProfOff() { c->prof = false; } } prof_off{ctx};
  char* p = ws;
  for (int l = 0; l < L; ++l) {
    cudaStream_t sf = ctx->lvl_stream[2 * l], sc = ctx->lvl_stream[2 * l + 1];
    const int nbl = level_batch(ctx, l, count[l], batch);
    char* q = p;
    uint64_t* ids = (uint64_t*)q; q += align256((size_t)nbl * 8);
    double* y = (double*)q; q += align256((size_t)nbl * ctx->lv[0].nodes * 8);
    double* y2 = (double*)q; q += align256((size_t)nbl * ctx->lv[0].nodes * 8);
    p += level_run_ws(ctx, l, nbl);
    if (count[l] == 0) continue;
    if ((r = order_after(ctx, st, sf)) != MLMC_OK) return r;
    ctx->prof_level = l;
    for (int64_t done = 0; done < count[l]; done += nbl) {
      int nb = (int)((count[l] - done) < nbl ? (count[l] - done) : nbl);
      CK(ctx, launch_iota((uint64_t)(first_id[l] + done), nb, ids, sf));
      ctx->launches += 1;
      if ((r = sample_level_into(ctx, l, seed, nullptr, ids, nullptr, nb, y, y2, nullptr, nullptr, nullptr,
                                 q, sf, sc)) != MLMC_OK)
        return r;
      if ((r = mlmc_accumulate(ctx, l, y, y2, nb, sf)) != MLMC_OK) return r;
    }
    if ((r = order_after(ctx, sf, st)) != MLMC_OK) return r;
  }
  return MLMC_OK;
}

static mlmc_status fill_stats(mlmc_ctx* ctx, double* stats) {
  unsigned long long cnt[N_COUNTERS];
  CK(ctx, cudaMemcpy(cnt, ctx->d_cnt, sizeof cnt, cudaMemcpyDeviceToHost));
  unsigned long long tot[6] = {0, 0, 0, 0, 0, 0};
  for (int l = 0; l < MLMC_MAX_LEVELS; ++l)
    for (int q = 0; q < 6; ++q) tot[q] += cnt[CNT_LEVEL + CNT_PER_LEVEL * l + q];
  if (stats) {
    double solve_ms = 0.0;
    for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
      float ms = 0.f;
      CK(ctx, cudaEventElapsedTime(&ms, ctx->ev_pool[i], ctx->ev_pool[i + 1]));
      solve_ms += ms;
    }
    stats[0] = solve_ms;
    stats[1] = (double)(ctx->ev_used / 2);
    stats[2] = (double)tot[1];
    stats[3] = (double)tot[2];
    stats[4] = (double)tot[3];
    stats[5] = (double)tot[4];
    stats[6] = (double)tot[0];
    stats[7] = (double)ctx->launches;
    stats[8] = (double)tot[5];
  }
  if (cnt[CNT_TC_TIMEOUT]) {
    char b[96];
    snprintf(b, sizeof b, "%llu KL tensor-core tiles timed out waiting for their MMAs", cnt[CNT_TC_TIMEOUT]);
    return fail(ctx, MLMC_ERR_TIMEOUT, b);
  }
  if (tot[0]) {
    char b[96];
    snprintf(b, sizeof b, "%llu sample solves did not converge", tot[0]);
    return fail(ctx, MLMC_ERR_NOT_CONVERGED, b);
  }
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_kl_info(const mlmc_ctx* ctx, int* rank, double* s_eff) {
  if (!ctx) return MLMC_ERR_ARG;
  if (rank) *rank = ctx->cfg.kl_kind == MLMC_KL_AFFINE_GAUSSIAN ? ctx->kl_rank : ctx->M;
  if (s_eff) *s_eff = ctx->cfg.kl_kind == MLMC_KL_AFFINE_GAUSSIAN ? ctx->kl_s_eff : 1.0;
  return MLMC_OK;
}

// Check of the bounded-wait path of the tensor-core KL kernel.
extern "C" mlmc_status mlmc_check_timeout_path(mlmc_ctx* ctx, long long polls) {
  if (!ctx) return MLMC_ERR_ARG;
  if (polls < -1) return fail(ctx, MLMC_ERR_ARG, "mlmc_check_timeout_path: polls must be >= -1");
  ctx->tc_check_limit = polls;
  return MLMC_OK;
}

// Per-level counters of the solves since the last reset and the solve-kernel
// device time of the last run call's launches of each level.
extern "C" mlmc_status mlmc_level_stats(mlmc_ctx* ctx, double* out) {
  if (!ctx || !out) return MLMC_ERR_ARG;
  unsigned long long cnt[N_COUNTERS];
  CK(ctx, cudaMemcpy(cnt, ctx->d_cnt, sizeof cnt, cudaMemcpyDeviceToHost));
  const int L = ctx->cfg.n_levels;
  for (int l = 0; l < L; ++l) {
    double* o = out + 8 * l;
    o[0] = 0.0;
    o[1] = 0.0;
    for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
      if (ctx->ev_grid[i / 2] != l) continue;
      float ms = 0.f;
      CK(ctx, cudaEventElapsedTime(&ms, ctx->ev_pool[i], ctx->ev_pool[i + 1]));
      o[0] += ms;
      o[1] += 1.0;
    }
    const unsigned long long* c = cnt + CNT_LEVEL + CNT_PER_LEVEL * l;
    o[2] = (double)c[1];   // CG iterations x nodes
    o[3] = (double)c[2];   // nonlinear iterations x nodes
    o[4] = (double)c[5];   // CG iterations x nodes in FP64
    o[5] = (double)c[3];   // truncations
    o[6] = (double)c[4];   // halvings / retried pseudo-steps
    o[7] = (double)c[0];   // non-converged solves
  }
  return MLMC_OK;
}

static mlmc_status run_begin(mlmc_ctx* ctx, void* stream) {
  mlmc_status r = mlmc_reset(ctx, stream);
  if (r != MLMC_OK) return r;
  ctx->ev_used = 0;
  ctx->ev_level.clear();
  ctx->ev_grid.clear();
  ctx->sync_used = 0;
  ctx->launches = 0;
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_run(mlmc_ctx* ctx, const int64_t* N_l, uint64_t seed, int batch,
                                void* ws, size_t ws_bytes, double* mean, double* var, double* V_l,
                                double* C_l, double* rmse, double* stats, void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  if (!N_l || batch < 1 || batch > 65535) return fail(ctx, MLMC_ERR_ARG, "mlmc_run: bad arguments");
  const int L = ctx->cfg.n_levels;
  for (int l = 0; l < L; ++l)
    if (N_l[l] < 0) return fail(ctx, MLMC_ERR_ARG, "mlmc_run: negative sample count");
  if (!check_ws(ctx, ws, ws_bytes, run_ws(ctx, N_l, batch))) return MLMC_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  mlmc_status r;
  if ((r = run_begin(ctx, stream)) != MLMC_OK) return r;
  int64_t first[MLMC_MAX_LEVELS] = {};
  double lvl_ms[MLMC_MAX_LEVELS];
  if ((r = run_levels(ctx, first, N_l, seed, batch, (char*)ws, st, lvl_ms)) != MLMC_OK) return r;
  if ((r = mlmc_estimate(ctx, mean, var, nullptr, nullptr, V_l, nullptr, rmse, stream)) != MLMC_OK) return r;
  for (int l = 0; l < L; ++l)
    if (C_l) C_l[l] = N_l[l] > 0 ? lvl_ms[l] * 1e-3 / (double)N_l[l] : 0.0;
  return fill_stats(ctx, stats);
}

extern "C" mlmc_status mlmc_run_more(mlmc_ctx* ctx, const int64_t* first_id, const int64_t* count,
                                     uint64_t seed, int batch, void* ws, size_t ws_bytes,
                                     double* solve_seconds, void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  if (!first_id || !count || batch < 1 || batch > 65535)
    return fail(ctx, MLMC_ERR_ARG, "mlmc_run_more: bad arguments");
  const int L = ctx->cfg.n_levels;
  for (int l = 0; l < L; ++l)
    if (count[l] < 0 || first_id[l] < 0) return fail(ctx, MLMC_ERR_ARG, "mlmc_run_more: negative id or count");
  if (!check_ws(ctx, ws, ws_bytes, run_ws(ctx, count, batch))) return MLMC_ERR_WORKSPACE;
  ctx->ev_used = 0;
  ctx->ev_level.clear();
  ctx->ev_grid.clear();
  ctx->sync_used = 0;
  double lvl_ms[MLMC_MAX_LEVELS];
  mlmc_status r = run_levels(ctx, first_id, count, seed, batch, (char*)ws, (cudaStream_t)stream, lvl_ms);
  if (r != MLMC_OK) return r;
  if (solve_seconds)
    for (int l = 0; l < L; ++l) solve_seconds[l] = lvl_ms[l] * 1e-3;
  return fill_stats(ctx, nullptr);
}

extern "C" mlmc_status mlmc_run_to_rmse(mlmc_ctx* ctx, double eps, const int64_t* N_pilot,
                                        int max_rounds, int64_t max_per_level, uint64_t seed,
                                        int batch, void* ws, size_t ws_bytes, int64_t* N_l,
                                        double* mean, double* var, double* V_l, double* C_l,
                                        double* rmse, double* bias, void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  const int L = ctx->cfg.n_levels;
  if (!(eps > 0.0) || !N_pilot || !N_l || max_rounds < 0 || max_per_level < 1 || batch < 1 ||
      batch > 65535)
    return fail(ctx, MLMC_ERR_ARG, "mlmc_run_to_rmse: bad arguments");
  int64_t cap[MLMC_MAX_LEVELS];
  for (int l = 0; l < L; ++l) {
    if (N_pilot[l] < 1) return fail(ctx, MLMC_ERR_ARG, "mlmc_run_to_rmse: every level needs a pilot sample");
    cap[l] = batch;
  }
  if (!check_ws(ctx, ws, ws_bytes, run_ws(ctx, cap, batch))) return MLMC_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  mlmc_status r;
  if ((r = run_begin(ctx, stream)) != MLMC_OK) return r;
  int64_t first[MLMC_MAX_LEVELS] = {}, cnt[MLMC_MAX_LEVELS];
  double lvl_ms[MLMC_MAX_LEVELS], ms_total[MLMC_MAX_LEVELS] = {}, V[MLMC_MAX_LEVELS], Cl[MLMC_MAX_LEVELS];
  for (int l = 0; l < L; ++l) { cnt[l] = N_pilot[l] < max_per_level ? N_pilot[l] : max_per_level; N_l[l] = 0; }
  // Giles' allocation (Operations Research 56, 2008): with variance V_l and
  // cost C_l per pair, N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k))
  // makes sum_l V_l / N_l <= eps^2 / 2 at least total cost.
  for (int round = 0;; ++round) {
    ctx->ev_used = 0;
    ctx->ev_level.clear();
    ctx->ev_grid.clear();
    ctx->sync_used = 0;
    if ((r = run_levels(ctx, first, cnt, seed, batch, (char*)ws, st, lvl_ms)) != MLMC_OK) return r;
    for (int l = 0; l < L; ++l) {
      N_l[l] += cnt[l];
      first[l] += cnt[l];
      ms_total[l] += lvl_ms[l];
    }
    if ((r = fill_stats(ctx, nullptr)) != MLMC_OK) return r;
    if ((r = mlmc_estimate(ctx, nullptr, nullptr, nullptr, nullptr, V, nullptr, nullptr, stream)) != MLMC_OK)
      return r;
    double S = 0.0;
    for (int l = 0; l < L; ++l) {
      Cl[l] = ms_total[l] * 1e-3 / (double)N_l[l];
      S += sqrt(V[l] * Cl[l]);
    }
    if (round >= max_rounds) break;
    int64_t more = 0;
    for (int l = 0; l < L; ++l) {
      double want = Cl[l] > 0.0 ? ceil(2.0 / (eps * eps) * sqrt(V[l] / Cl[l]) * S) : (double)N_l[l];
      int64_t target = want > (double)max_per_level ? max_per_level : (int64_t)want;
      cnt[l] = target > N_l[l] ? target - N_l[l] : 0;
      more += cnt[l];
    }
    if (more == 0) break;
  }
  double b = 0.0;
  if ((r = estimate_impl(ctx, mean, var, nullptr, nullptr, V_l, nullptr, rmse, &b, stream)) != MLMC_OK)
    return r;
  if (bias) *bias = b;
  if (C_l)
    for (int l = 0; l < L; ++l) C_l[l] = Cl[l];
  // The allocation drives the sampling error to eps^2 / 2; the target
  // sum_l V_l / N_l + bias^2 <= eps^2 also needs bias^2 <= eps^2 / 2, which no
  // sample count changes on a fixed hierarchy.
  if (b * b > 0.5 * eps * eps) {
    char m[200];
    snprintf(m, sizeof m, "mlmc_run_to_rmse: sampling error at target, but the bias estimate %.4g "
             "exceeds eps/sqrt(2) = %.4g: eps is not reached with %d levels", b, eps / sqrt(2.0), L);
    ctx->err = m;
    return MLMC_WARN_BIAS;
  }
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_diagnostics(mlmc_ctx* ctx, double* mean_norm, double* alpha,
                                        double* censored, void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  const int L = ctx->cfg.n_levels;
  const int64_t n0 = ctx->lv[0].nodes;
  std::vector<double> mean_l((size_t)L * n0);
  mlmc_status r = estimate_impl(ctx, nullptr, nullptr, mean_l.data(), nullptr, nullptr, nullptr,
                                nullptr, nullptr, stream);
  if (r != MLMC_OK) return r;
  unsigned long long cnt[N_COUNTERS];
  CK(ctx, cudaMemcpy(cnt, ctx->d_cnt, sizeof cnt, cudaMemcpyDeviceToHost));
  // level-0 lumped mass: cell volume times 1/2 per axis on which the node is
  // on the boundary
  const LevelDesc& l0 = ctx->lv[0];
  std::vector<double> nrm(L, 0.0);
  for (int64_t A = 0; A < n0; ++A) {
    const int64_t i = A % l0.N[0], j = (A / l0.N[0]) % l0.N[1], k = A / ((int64_t)l0.N[0] * l0.N[1]);
    double w = l0.vol;
    if (i == 0 || i == l0.n[0]) w *= 0.5;
    if (j == 0 || j == l0.n[1]) w *= 0.5;
    if (l0.dim == 3 && (k == 0 || k == l0.n[2])) w *= 0.5;
    for (int l = 0; l < L; ++l) nrm[l] += w * mean_l[(size_t)l * n0 + A] * mean_l[(size_t)l * n0 + A];
  }
  for (int l = 0; l < L; ++l) {
    nrm[l] = sqrt(nrm[l]);
    if (mean_norm) mean_norm[l] = nrm[l];
    if (censored)
      censored[l] = ctx->N_acc[l] > 0 ? (double)cnt[CNT_CENSORED + l] / ((double)ctx->N_acc[l] * (double)n0)
                                      : 0.0;
  }
  if (alpha) {
    // least-squares slope of -log2 ||mean(Y_l)|| over the correction levels l >= 1
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    int m = 0;
    for (int l = 1; l < L; ++l) {
      if (!(nrm[l] > 0.0)) continue;
      const double y = -log2(nrm[l]);
      sx += l; sy += y; sxx += (double)l * l; sxy += l * y; ++m;
    }
    *alpha = m >= 2 ? (m * sxy - sx * sy) / (m * sxx - sx * sx) : NAN;
  }
  return MLMC_OK;
}

// ----------------------------------------------------------------- state
extern "C" mlmc_status mlmc_get_state(mlmc_ctx* ctx, int64_t* N_l, double* mean_l, double* m2_l,
                                      double* mean2_l, void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  const int L = ctx->cfg.n_levels;
  const int64_t n0 = ctx->lv[0].nodes;
  cudaStream_t st = (cudaStream_t)stream;
  double* out[3] = {mean_l, m2_l, mean2_l};
  for (int q = 0; q < 3; ++q)
    if (out[q])
      CK(ctx, cudaMemcpyAsync(out[q], ctx->d_acc + (int64_t)q * L * n0, sizeof(double) * L * n0,
                              cudaMemcpyDeviceToHost, st));
  CK(ctx, cudaStreamSynchronize(st));
  if (N_l)
    for (int l = 0; l < L; ++l) N_l[l] = ctx->N_acc[l];
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_set_state(mlmc_ctx* ctx, const int64_t* N_l, const double* mean_l,
                                      const double* m2_l, const double* mean2_l, void* stream) {
  if (!ctx) return MLMC_ERR_ARG;
  if (!N_l || !mean_l || !m2_l || !mean2_l) return fail(ctx, MLMC_ERR_ARG, "mlmc_set_state: NULL input");
  const int L = ctx->cfg.n_levels;
  const int64_t n0 = ctx->lv[0].nodes;
  for (int l = 0; l < L; ++l)
    if (N_l[l] < 0) return fail(ctx, MLMC_ERR_ARG, "mlmc_set_state: negative count");
  cudaStream_t st = (cudaStream_t)stream;
  const double* in[3] = {mean_l, m2_l, mean2_l};
  for (int q = 0; q < 3; ++q)
    CK(ctx, cudaMemcpyAsync(ctx->d_acc + (int64_t)q * L * n0, in[q], sizeof(double) * L * n0,
                            cudaMemcpyHostToDevice, st));
  CK(ctx, cudaStreamSynchronize(st));
  for (int l = 0; l < L; ++l) ctx->N_acc[l] = N_l[l];
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_merge_states(int levels, int64_t nodes0, int64_t* N_a, double* mean_a,
                                         double* m2_a, double* mean2_a, const int64_t* N_b,
                                         const double* mean_b, const double* m2_b,
                                         const double* mean2_b) {
  if (levels < 1 || levels > MLMC_MAX_LEVELS || nodes0 < 1 || !N_a || !mean_a || !m2_a || !mean2_a ||
      !N_b || !mean_b || !m2_b || !mean2_b)
    return MLMC_ERR_ARG;
  for (int l = 0; l < levels; ++l) {
    const int64_t na = N_a[l], nb = N_b[l];
    if (na < 0 || nb < 0) return MLMC_ERR_ARG;
    if (nb == 0) continue;
    const int64_t off = (int64_t)l * nodes0;
    if (na == 0) {
      for (int64_t i = 0; i < nodes0; ++i) {
        mean_a[off + i] = mean_b[off + i];
        m2_a[off + i] = m2_b[off + i];
        mean2_a[off + i] = mean2_b[off + i];
      }
    } else {
      const double dna = (double)na, dnb = (double)nb, nt = dna + dnb;
      for (int64_t i = 0; i < nodes0; ++i) {
        const double delta = mean_b[off + i] - mean_a[off + i];
        mean_a[off + i] += delta * dnb / nt;
        m2_a[off + i] += m2_b[off + i] + delta * delta * dna * dnb / nt;
        mean2_a[off + i] += (mean2_b[off + i] - mean2_a[off + i]) * dnb / nt;
      }
    }
    N_a[l] = na + nb;
  }
  return MLMC_OK;
}
