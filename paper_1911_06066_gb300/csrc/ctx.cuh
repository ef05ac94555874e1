// Internal view of the context shared by the C ABI translation units
// (abi.cu: setup, steps and whole runs; serve.cu: the request server).
#pragma once
#include <string>
#include <vector>

#include "internal.cuh"

struct mlmc_ctx {
  mlmc_config cfg;
  int device;
  mlmc::LevelDesc lv[MLMC_MAX_LEVELS];
  mlmc::Physics ph;
  mlmc::SolverParams sp;
  int M;
  double* d_sqrt_lam = nullptr;
  int* d_idx = nullptr;
  double* d_phi[MLMC_MAX_LEVELS][3] = {};
  float* d_phi32[MLMC_MAX_LEVELS][3] = {};   // FP32 copies (tensor-core KL synthesis)
  // the paper's KL variant (kl_kind 1): per level the mode table [cells][M]
  // (FP64 and FP32), the pivots and pivot rows of the factor, the rank, s_eff
  double* d_tab64[MLMC_MAX_LEVELS] = {};
  float* d_tab32[MLMC_MAX_LEVELS] = {};
  double* d_xp = nullptr;
  double* d_lpiv = nullptr;
  int kl_rank = 0;
  double kl_s_eff = 0.0;
  double* d_acc = nullptr;        // [3][levels][nodes0]: mean, M2, mean of Y2
  int64_t* d_N = nullptr;         // [levels]
  double* d_est = nullptr;        // estimate output
  unsigned long long* d_cnt = nullptr;  // solver counters (see N_COUNTERS)
  int64_t N_acc[MLMC_MAX_LEVELS] = {};
  // streams for concurrent solves: [2l] fine / [2l+1] coarse solves of level
  // l inside mlmc_run; aux_pub for the coarse solve of mlmc_sample_level
  cudaStream_t lvl_stream[2 * MLMC_MAX_LEVELS] = {};
  cudaStream_t aux_pub = nullptr;
  std::vector<cudaEvent_t> sync_pool;   // ordering-only events
  size_t sync_used = 0;
  // launch accounting and solve-kernel timing, active inside mlmc_run
  bool prof = false;
  long launches = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_level;    // level pair of each (start, end) event pair
  std::vector<int> ev_grid;     // grid level of the solve it brackets
  int prof_level = 0;
  size_t ev_used = 0;
  // per-level solver layout chosen by mlmc_autotune: 0 = the smallest
  // cluster that holds a sample, C > 0 = clusters of C CTAs, -1 = the
  // block-per-sample kernel
  int tuned_C[MLMC_MAX_LEVELS] = {};
  // CUDA-graph form of the run schedule (cfg.use_graph): true while a run's
  // launches are being captured; the instantiated graph of the last run, kept
  // for in-place updates; how many runs were launched as a graph
  bool capturing = false;
  cudaGraphExec_t graph_exec = nullptr;
  long graph_runs = 0;
  long long tc_check_limit = -1;   // mlmc_check_timeout_path: -1 normal operation
  // group-layout solves of one context run one after another (each waits for
  // the previous one): grp_ev is recorded after every group launch and is
  // valid for the next one while grp_ev_valid holds (reset at the start and
  // end of a graph capture, whose events cannot be waited on across it)
  cudaEvent_t grp_ev = nullptr;
  bool grp_ev_valid = false;
  std::string err;
};

namespace mlmc {
mlmc_status fail(mlmc_ctx* ctx, mlmc_status st, const std::string& msg);
mlmc_status cuda_fail(mlmc_ctx* ctx, cudaError_t e, const char* where);
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct PairWs {
  size_t xi, kl, Zf, Zc, tf, tc, info, solve_f, solve_c, total;
};
// Workspace of n level-l pairs (xi, both fields, both activation maps, info
// and the two solves' scratch), 256-byte aligned offsets.
PairWs pair_ws(const mlmc_ctx* c, int level, int n);
// Makes `waiter` wait for the work enqueued so far on `src`.
mlmc_status order_after(mlmc_ctx* ctx, cudaStream_t src, cudaStream_t waiter);
// n level-l pairs: xi (one seed, or seeds[n] per sample), fields, the fine
// solve on st_f and the coarse one on st_c, the difference on the coarsest
// grid into y, y2.  stim (device [n][3] or NULL) overrides the stimulus
// centre per sample.  t_fine / t_coarse / info may be NULL.
mlmc_status sample_level_into(mlmc_ctx* ctx, int level, uint64_t seed, const uint64_t* seeds,
                              const uint64_t* ids, const double* stim, int n, double* y, double* y2,
                              double* t_fine, double* t_coarse, mlmc_sample_info* info, char* ws,
                              cudaStream_t st_f, cudaStream_t st_c);
// mlmc_estimate plus the bias estimate (synchronises the stream).
mlmc_status estimate_impl(mlmc_ctx* ctx, double* mean, double* var, double* mean_l, double* var_l,
                          double* V_l, int64_t* N_l, double* rmse, double* bias, void* stream);
}  // namespace mlmc

#define CK(ctx, expr)                                        \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #expr); \
  } while (0)
