// mlmc_solve_noalloc: the per-sample solve of mlmc_solve for callers that may
// not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc (or any allocator) is off
// limits -- for instance inside a region whose memory budget was fixed up
// front by a host framework, in a plugin that must not touch the device heap,
// or where an allocation could synchronise the device at the wrong moment.
// Such a caller still owns its inputs (Z) and outputs (t_act, info) but cannot
// provide the solver's workspace.  This entry point therefore takes its
// scratch from one file-scope device array, allocated once when the module is
// loaded and held by every device that loads the library until the process
// exits.  It calls no cudaMalloc / cudaFree and no allocating library routine.
//
// The kernels are the ones mlmc_solve launches (coupling assembly and the
// Newton-CG sweep); only the origin of the scratch differs.
#include <math.h>
#include <stdio.h>

#include <mutex>
#include <string>

#include "internal.cuh"

namespace mlmc {
void set_create_error(const std::string& msg);  // abi.cu: text for mlmc_last_error(NULL)
}

using namespace mlmc;

// Scratch shared by every call on a device: MLMC_NOALLOC_SCRATCH_BYTES.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MLMC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (in host code the array's name is only a host-side stand-in).  The
// same one-time set-up loads the modules of every kernel this entry point
// launches (CUDA loads modules lazily by default: without this, the first
// launch of each would load it, and the array itself is placed on the device
// when this module loads), so that every later call only enqueues work.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    LevelDesc probe = {};
    for (int dim = 2; dim <= 3 && e == cudaSuccess; ++dim) {
      probe.dim = dim;
      e = preload_solve(probe, false);
      if (e == cudaSuccess) e = preload_solve(probe, true);
    }
    if (e == cudaSuccess) e = preload_assemble();
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

mlmc_status reject(mlmc_status st, const std::string& msg) {
  set_create_error("mlmc_solve_noalloc: " + msg);
  return st;
}

}  // namespace

extern "C" mlmc_status mlmc_solve_noalloc(const mlmc_config* cfg, int level, const double* Z,
                                          int n, double* t_act, mlmc_sample_info* info,
                                          void* stream) {
  if (!cfg) return reject(MLMC_ERR_ARG, "cfg is NULL");
  const mlmc_config& c = *cfg;
  if (c.dim < 1 || c.dim > 3) return reject(MLMC_ERR_ARG, "dim must be 1, 2 or 3");
  if (level < 0 || level >= c.n_levels || c.n_levels > MLMC_MAX_LEVELS)
    return reject(MLMC_ERR_ARG, "level out of range");
  if (!(c.kl_sigma2 >= 0.0) || c.precond < MLMC_PRECOND_JACOBI || c.precond > MLMC_PRECOND_GMG)
    return reject(MLMC_ERR_ARG, "invalid configuration");
  if (c.m0 < 1 || !(c.T > 0.0) || !(c.newton_tol > 0.0) || c.newton_max < 1 ||
      !(c.lin_rtol > 0.0) || c.lin_max < 1 || !(c.s_t > 0.0) || !(c.s_l0 > 0.0))
    return reject(MLMC_ERR_ARG, "invalid configuration");
  if (c.precision != MLMC_PREC_FP64 && c.precision != MLMC_PREC_MIXED)
    return reject(MLMC_ERR_ARG, "unknown precision");
  if (!model_config_ok(c)) return reject(MLMC_ERR_ARG, "time scheme, stimulus or QoI out of range");
  if (n < 0 || n > 65535 || (n > 0 && (!Z || !t_act))) return reject(MLMC_ERR_ARG, "bad arguments");

  // level geometry and parameters, derived by the same helpers as mlmc_create
  // and mlmc_solve
  LevelDesc lv;
  std::string why;
  if (!derive_level(c, level, &lv, &why)) return reject(MLMC_ERR_ARG, why);
  Physics ph;
  derive_physics(c, &ph);
  const bool mixed = level_mixed(c, lv);
  const SolverParams sp = level_solver_params(c, lv, mixed);

  // The scratch is mlmc_solve's workspace layout carved from the static array.
  // Bound the per-sample size first, so that no product below can wrap.
  const size_t per_sample_floor = (size_t)lv.nodes * n_offsets(c.dim) * 8;   // FP64 couplings alone
  if (n > 0 && (size_t)n > (size_t)MLMC_NOALLOC_SCRATCH_BYTES / per_sample_floor) {
    char b[200];
    snprintf(b, sizeof b, "%d samples of level %d need more than %zu bytes of scratch; the static "
             "scratch holds %zu bytes (MLMC_NOALLOC_SCRATCH_BYTES)", n, level,
             (size_t)MLMC_NOALLOC_SCRATCH_BYTES, (size_t)MLMC_NOALLOC_SCRATCH_BYTES);
    return reject(MLMC_ERR_WORKSPACE, b);
  }
  const SolveWs w = solve_ws(c, lv, n, mixed);
  if (w.total > (size_t)MLMC_NOALLOC_SCRATCH_BYTES) {
    char b[200];
    snprintf(b, sizeof b, "%d samples of level %d need %zu bytes of scratch; the static scratch "
             "holds %zu bytes (MLMC_NOALLOC_SCRATCH_BYTES)", n, level, w.total,
             (size_t)MLMC_NOALLOC_SCRATCH_BYTES);
    return reject(MLMC_ERR_WORKSPACE, b);
  }
  if (n == 0) return MLMC_OK;

  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return reject(MLMC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  char* ws = (char*)base;
  cudaStream_t st = (cudaStream_t)stream;
  // Every scratch word the kernels read is written earlier in the same call
  // (couplings by the assembly, states, residuals and CG vectors by the sweep),
  // so the previous call's contents need no clearing.
  double* coef64 = (double*)(ws + w.coef64);
  float* coef32 = mixed ? (float*)(ws + w.coef32) : nullptr;
  e = launch_assemble(lv, ph, Z, n, coef64, coef32, st);
  if (e == cudaSuccess)
    e = launch_solve(lv, ph, sp, mixed, n, coef64, coef32, nullptr, (double*)(ws + w.ubuf),
                     (double*)(ws + w.F), (double*)(ws + w.Ku), (double*)(ws + w.Kd),
                     (void*)(ws + w.kr), t_act, info, nullptr, st);
  if (e != cudaSuccess) return reject(MLMC_ERR_CUDA, cudaGetErrorString(e));
  return MLMC_OK;
}
