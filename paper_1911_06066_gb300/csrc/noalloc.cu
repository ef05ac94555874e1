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

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch on the current device, looked up once per
// device (in host code the array's name is only a host-side stand-in).
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
  if (c.dim != 2 && c.dim != 3) return reject(MLMC_ERR_ARG, "dim must be 2 or 3");
  if (level < 0 || level >= c.n_levels || c.n_levels > MLMC_MAX_LEVELS)
    return reject(MLMC_ERR_ARG, "level out of range");
  if (c.m0 < 1 || !(c.T > 0.0) || !(c.newton_tol > 0.0) || c.newton_max < 1 ||
      !(c.lin_rtol > 0.0) || c.lin_max < 1 || !(c.s_t > 0.0) || !(c.s_l0 > 0.0))
    return reject(MLMC_ERR_ARG, "invalid configuration");
  if (c.precision != MLMC_PREC_FP64 && c.precision != MLMC_PREC_MIXED)
    return reject(MLMC_ERR_ARG, "unknown precision");
  if (n < 0 || n > 65535 || (n > 0 && (!Z || !t_act))) return reject(MLMC_ERR_ARG, "bad arguments");

  // level geometry and parameters, as mlmc_create derives them
  const double pi = 3.141592653589793238462643;
  LevelDesc lv;
  lv.dim = c.dim;
  int64_t nodes = 1, cells = 1;
  double vol = 1.0;
  for (int d = 0; d < 3; ++d) {
    if (d < c.dim) {
      if (c.n0[d] < 1 || !(c.L[d] > 0.0)) return reject(MLMC_ERR_ARG, "invalid grid");
      int64_t nn = (int64_t)c.n0[d] << level;
      if (nn > (1 << 20)) return reject(MLMC_ERR_ARG, "grid too large");
      lv.n[d] = (int)nn; lv.N[d] = (int)nn + 1; lv.h[d] = c.L[d] / (double)nn;
    } else {
      lv.n[d] = 1; lv.N[d] = 1; lv.h[d] = 1.0;
    }
    nodes *= lv.N[d]; cells *= lv.n[d]; vol *= (d < c.dim ? lv.h[d] : 1.0);
  }
  lv.nodes = nodes; lv.cells = cells; lv.vol = vol;
  lv.m = (int)((int64_t)c.m0 << level);
  lv.T = c.T;
  lv.dt = c.T / (double)lv.m;
  Physics ph;
  ph.c = c.c; ph.a = c.a; ph.s_t = c.s_t; ph.s_l0 = c.s_l0;
  ph.th0 = c.theta0_deg * pi / 180.0;
  ph.th1 = c.theta1_deg * pi / 180.0;
  ph.Lz = c.dim == 3 ? c.L[2] : 1.0;
  ph.stim_r2 = c.stim_r * c.stim_r;
  for (int d = 0; d < 3; ++d) ph.stim_c[d] = c.stim_c[d];
  ph.stim_ps = nullptr;
  // FP32 inner solves only where c dt max r' <= mixed_cdr_max, as in mlmc_solve
  const double rmax = c.c * ((1.0 + c.a) * (1.0 + c.a) / 3.0 - c.a);
  const double cdr_lim = c.mixed_cdr_max > 0.0 ? c.mixed_cdr_max : 2.0;
  const bool mixed = c.precision == MLMC_PREC_MIXED && lv.dt * rmax <= cdr_lim;
  SolverParams sp;
  sp.newton_tol = c.newton_tol;
  sp.newton_max = c.newton_max;
  sp.lin_rtol = mixed ? fmax(c.lin_rtol, 1e-5) : c.lin_rtol;
  sp.lin_max = c.lin_max;
  sp.ls_full_step = 1e-6;
  sp.step_max = step_limit(c.c, c.a, lv.dt);
  sp.cg_scale = 0;   // the block kernel does not scale

  // scratch layout of mlmc_solve's workspace, carved from the static array
  size_t N = (size_t)nodes, NO = (size_t)n_offsets(c.dim), kr = mixed ? 4 : 8;
  size_t o_coef64 = 0;
  size_t o_coef32 = o_coef64 + al256((size_t)n * NO * N * 8);
  size_t o_ubuf = o_coef32 + (mixed ? al256((size_t)n * NO * N * 4) : 0);
  size_t o_F = o_ubuf + al256((size_t)n * 2 * N * 8);
  size_t o_Ku = o_F + al256((size_t)n * N * 8);
  size_t o_Kd = o_Ku + al256((size_t)n * N * 8);
  size_t o_kr = o_Kd + al256((size_t)n * N * 8);
  size_t need = o_kr + al256((size_t)n * 7 * N * kr);
  if (need > (size_t)MLMC_NOALLOC_SCRATCH_BYTES) {
    char b[200];
    snprintf(b, sizeof b, "%d samples of level %d need %zu bytes of scratch; the static scratch "
             "holds %zu bytes (MLMC_NOALLOC_SCRATCH_BYTES)", n, level, need,
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
  double* coef64 = (double*)(ws + o_coef64);
  float* coef32 = mixed ? (float*)(ws + o_coef32) : nullptr;
  e = launch_assemble(lv, ph, Z, n, coef64, coef32, st);
  if (e == cudaSuccess)
    e = launch_solve(lv, ph, sp, mixed, n, coef64, coef32, nullptr, (double*)(ws + o_ubuf),
                     (double*)(ws + o_F), (double*)(ws + o_Ku), (double*)(ws + o_Kd),
                     (void*)(ws + o_kr), t_act, info, nullptr, st);
  if (e != cudaSuccess) return reject(MLMC_ERR_CUDA, cudaGetErrorString(e));
  return MLMC_OK;
}
