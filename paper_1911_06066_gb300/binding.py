"""Thin Python binding of the C ABI in ``include/mlmc.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library ``lib/libmlmc_gb300.so``.  Device memory and streams come from
PyTorch (tensors' ``data_ptr()`` and ``torch.cuda.current_stream()``).  If the
library is missing the import of this module still works, but every call
raises -- there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmlmc_gb300.so")

MLMC_MAX_LEVELS = 8
MLMC_OK = 0
MLMC_WARN_BIAS = 1
MLMC_PREC_FP64 = 0
MLMC_PREC_MIXED = 1
STATUS = {0: "MLMC_OK", -1: "MLMC_ERR_ARG", -2: "MLMC_ERR_OOM", -3: "MLMC_ERR_NOT_CONVERGED",
          -4: "MLMC_ERR_TIMEOUT", -5: "MLMC_ERR_CUDA", -6: "MLMC_ERR_WORKSPACE"}


class mlmc_config(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_levels", C.c_int), ("n0", C.c_int * 3), ("m0", C.c_int),
                ("L", C.c_double * 3), ("T", C.c_double), ("c", C.c_double), ("a", C.c_double),
                ("s_t", C.c_double), ("s_l0", C.c_double), ("theta0_deg", C.c_double),
                ("theta1_deg", C.c_double), ("stim_r", C.c_double), ("stim_c", C.c_double * 3),
                ("kl_sigma2", C.c_double), ("kl_ell", C.c_double), ("kl_modes", C.c_int),
                ("precision", C.c_int), ("newton_tol", C.c_double), ("newton_max", C.c_int),
                ("lin_rtol", C.c_double), ("lin_max", C.c_int), ("solver", C.c_int),
                ("mixed_cdr_max", C.c_double), ("cluster_size", C.c_int), ("precond", C.c_int),
                ("mg_nu", C.c_int), ("mg_coarse_sweeps", C.c_int), ("use_graph", C.c_int),
                ("time_scheme", C.c_int), ("stim_kind", C.c_int), ("stim_amp", C.c_double),
                ("stim_sigma", C.c_double), ("stim_t1", C.c_double), ("qoi", C.c_int),
                ("kl_kind", C.c_int), ("kl_tol", C.c_double), ("kl_s", C.c_double),
                ("kl_delta", C.c_double), ("kl_cand_n", C.c_int * 3)]


MLMC_SOLVER_AUTO, MLMC_SOLVER_BLOCK, MLMC_SOLVER_CLUSTER = 0, 1, 2
MLMC_PRECOND_JACOBI, MLMC_PRECOND_GMG = 0, 1
MLMC_LAYOUT_GROUP = 200
MLMC_SCHEME_IE, MLMC_SCHEME_CN = 0, 1
MLMC_STIM_BALL, MLMC_STIM_PULSE = 0, 1
MLMC_QOI_ACTIVATION, MLMC_QOI_FINAL_STATE = 0, 1
MLMC_KL_SEPARABLE_EXP, MLMC_KL_AFFINE_GAUSSIAN = 0, 1


class mlmc_sample_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("failed_step", C.c_int32), ("newton_iters", C.c_int32),
                ("cg_iters", C.c_int32), ("truncations", C.c_int32), ("halvings", C.c_int32),
                ("max_newton", C.c_int32), ("pad", C.c_int32)]


INFO_FIELDS = [f[0] for f in mlmc_sample_info._fields_ if f[0] != "pad"]


class mlmc_server_config(C.Structure):
    _fields_ = [("max_batch", C.c_int), ("slots", C.c_int), ("mem_budget", C.c_size_t),
                ("keep_maps", C.c_int), ("max_wait_s", C.c_double)]


class mlmc_request(C.Structure):
    _fields_ = [("tag", C.c_int64), ("level", C.c_int), ("pad", C.c_int), ("seed", C.c_uint64),
                ("sample_id", C.c_uint64), ("stim_c", C.c_double * 3)]


class mlmc_result(C.Structure):
    _fields_ = [("tag", C.c_int64), ("level", C.c_int), ("status", C.c_int),
                ("newton_iters", C.c_int), ("cg_iters", C.c_int), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double)]

_lib = None


class MLMCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing; run __graft_entry__.build() "
                               "(there is no CPU fallback)" % LIB_PATH)
        l = C.CDLL(LIB_PATH)
        vp, i64, i32, u64, sz = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64, C.c_size_t
        ip = C.c_int
        sig = {
            "mlmc_create": ([C.POINTER(mlmc_config), C.POINTER(vp)], ip),
            "mlmc_destroy": ([vp], None),
            "mlmc_last_error": ([vp], C.c_char_p),
            "mlmc_level_info": ([vp, ip, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32)], ip),
            "mlmc_workspace_bytes": ([vp, ip, ip, C.POINTER(sz)], ip),
            "mlmc_xi": ([vp, u64, ip, vp, ip, vp, vp], ip),
            "mlmc_kl_field": ([vp, ip, vp, ip, vp, vp], ip),
            "mlmc_kl_tc_workspace_bytes": ([vp, ip, C.POINTER(sz)], ip),
            "mlmc_kl_field_tc": ([vp, ip, vp, ip, vp, vp, sz, vp], ip),
            "mlmc_solve": ([vp, ip, vp, ip, vp, vp, vp, vp, sz, vp], ip),
            "mlmc_slab_residual": ([vp, ip, vp, vp, ip, vp, vp, vp], ip),
            "mlmc_activation": ([vp, ip, vp, ip, vp, vp], ip),
            "mlmc_sample_level": ([vp, ip, u64, vp, ip, vp, vp, vp, vp, vp, vp, sz, vp], ip),
            "mlmc_accumulate": ([vp, ip, vp, vp, ip, vp], ip),
            "mlmc_reset": ([vp, vp], ip),
            "mlmc_estimate": ([vp, vp, vp, vp, vp, vp, vp, vp, vp], ip),
            "mlmc_run": ([vp, vp, u64, ip, vp, sz, vp, vp, vp, vp, vp, vp, vp], ip),
            "mlmc_run_workspace_bytes": ([vp, vp, ip, C.POINTER(sz)], ip),
            "mlmc_run_more": ([vp, vp, vp, u64, ip, vp, sz, vp, vp], ip),
            "mlmc_run_to_rmse": ([vp, C.c_double, vp, ip, i64, u64, ip, vp, sz, vp, vp, vp, vp, vp,
                                  vp, vp, vp], ip),
            "mlmc_diagnostics": ([vp, vp, vp, vp, vp], ip),
            "mlmc_level_stats": ([vp, vp], ip),
            "mlmc_check_timeout_path": ([vp, C.c_longlong], ip),
            "mlmc_kl_info": ([vp, C.POINTER(ip), C.POINTER(C.c_double)], ip),
            "mlmc_get_state": ([vp, vp, vp, vp, vp, vp], ip),
            "mlmc_set_state": ([vp, vp, vp, vp, vp, vp], ip),
            "mlmc_merge_states": ([ip, i64, vp, vp, vp, vp, vp, vp, vp, vp], ip),
            "mlmc_autotune": ([vp, ip, u64, vp, ip, vp, sz, C.POINTER(ip), vp, vp], ip),
            "mlmc_get_layout": ([vp, ip, C.POINTER(ip)], ip),
            "mlmc_set_layout": ([vp, ip, ip], ip),
            "mlmc_server_create": ([vp, C.POINTER(mlmc_server_config), C.POINTER(vp)], ip),
            "mlmc_server_submit": ([vp, vp, ip], ip),
            "mlmc_server_poll": ([vp, vp, ip, C.POINTER(ip), vp, vp, i64, C.c_double], ip),
            "mlmc_server_drain": ([vp, C.c_double], ip),
            "mlmc_server_stats": ([vp, vp], ip),
            "mlmc_server_clock": ([vp, C.POINTER(C.c_double)], ip),
            "mlmc_server_estimate": ([vp, vp, vp, vp, vp, vp, vp], ip),
            "mlmc_server_error": ([vp], C.c_char_p),
            "mlmc_server_destroy": ([vp], None),
            "mlmc_solve_noalloc": ([C.POINTER(mlmc_config), ip, vp, ip, vp, vp, vp], ip),
            "mlmc_probe_fma_rate": ([ip, vp, sz, C.POINTER(C.c_double), vp], ip),
        }
        for name, (args, res) in sig.items():
            f = getattr(l, name)
            f.argtypes = args
            f.restype = res
        _lib = l
    return _lib


def exported_symbols():
    """Names of the C-ABI functions this binding declares."""
    return ["mlmc_create", "mlmc_destroy", "mlmc_last_error", "mlmc_level_info",
            "mlmc_workspace_bytes", "mlmc_xi", "mlmc_kl_field", "mlmc_kl_tc_workspace_bytes",
            "mlmc_kl_field_tc", "mlmc_solve",
            "mlmc_slab_residual",
            "mlmc_activation", "mlmc_sample_level", "mlmc_accumulate", "mlmc_reset",
            "mlmc_estimate", "mlmc_run", "mlmc_run_workspace_bytes", "mlmc_run_more",
            "mlmc_run_to_rmse", "mlmc_diagnostics", "mlmc_level_stats", "mlmc_check_timeout_path", "mlmc_kl_info", "mlmc_get_state", "mlmc_set_state", "mlmc_merge_states",
            "mlmc_autotune", "mlmc_get_layout", "mlmc_set_layout", "mlmc_server_create",
            "mlmc_server_submit", "mlmc_server_poll", "mlmc_server_drain", "mlmc_server_stats",
            "mlmc_server_clock", "mlmc_server_estimate", "mlmc_server_error",
            "mlmc_server_destroy", "mlmc_solve_noalloc", "mlmc_probe_fma_rate"]


def fma_rate(fp64=True, stream=None):
    """Measured FMA rate of the current device in TFLOP/s (mlmc_probe_fma_rate)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = torch.empty(16 * 256 * 8 * sms, dtype=torch.uint8, device="cuda")
    r = C.c_double()
    st = lib().mlmc_probe_fma_rate(1 if fp64 else 0, C.c_void_p(out.data_ptr()), out.numel(),
                                   C.byref(r), _stream(stream))
    if st != MLMC_OK:
        raise MLMCError(st, lib().mlmc_last_error(None).decode())
    return r.value


def _dp(a):
    return a.ctypes.data_as(C.c_void_p)


class State:
    """Host copy of a context's accumulator state: per level the sample count
    ``N`` [L], running mean ``mean`` [L][nodes_0] and sum of squared
    deviations ``m2`` of the injected difference Y_l, and the running mean
    ``mean2`` of t_l^2 - t_{l-1}^2."""

    def __init__(self, N, mean, m2, mean2):
        self.N = np.ascontiguousarray(N, np.int64)
        self.mean = np.ascontiguousarray(mean, np.float64)
        self.m2 = np.ascontiguousarray(m2, np.float64)
        self.mean2 = np.ascontiguousarray(mean2, np.float64)

    @classmethod
    def empty(cls, levels, nodes0):
        z = np.zeros((levels, nodes0))
        return cls(np.zeros(levels, np.int64), z, z.copy(), z.copy())

    def as_array(self):
        """One flat float64 vector (counts first) for a collective or a file."""
        return np.concatenate([self.N.astype(np.float64), self.mean.ravel(), self.m2.ravel(),
                               self.mean2.ravel()])

    @classmethod
    def from_array(cls, a, levels, nodes0):
        a = np.asarray(a, np.float64)
        k = levels * nodes0
        N = np.rint(a[:levels]).astype(np.int64)
        r = a[levels:]
        return cls(N, r[:k].reshape(levels, nodes0), r[k:2 * k].reshape(levels, nodes0),
                   r[2 * k:3 * k].reshape(levels, nodes0))

    def merge(self, other):
        """In place: self <- self merged with other (mlmc_merge_states, on the CPU)."""
        L, n0 = self.mean.shape
        st = lib().mlmc_merge_states(L, n0, _dp(self.N), _dp(self.mean), _dp(self.m2),
                                     _dp(self.mean2), _dp(other.N), _dp(other.mean), _dp(other.m2),
                                     _dp(other.mean2))
        if st != MLMC_OK:
            raise MLMCError(st, "mlmc_merge_states")
        return self


def make_config(w, precision=MLMC_PREC_FP64, newton_tol=1e-12, newton_max=5000, lin_rtol=1e-12,
                lin_max=5000, levels=None, solver=MLMC_SOLVER_AUTO, mixed_cdr_max=None,
                cluster_size=0, precond=MLMC_PRECOND_JACOBI, mg_nu=0, mg_coarse_sweeps=0,
                use_graph=False):
    """mlmc_config from a workload dictionary (see workloads.py).

    precision: MLMC_PREC_FP64 or MLMC_PREC_MIXED (FP32 inner solves and the
    tensor-core KL field on levels with c dt max r' <= mixed_cdr_max).
    solver / cluster_size: kernel layout of the per-sample sweep.
    precond: MLMC_PRECOND_JACOBI or MLMC_PRECOND_GMG (geometric multigrid on
    levels whose step Hessians are positive definite; mg_nu / mg_coarse_sweeps
    its smoothing counts, 0 = defaults).  use_graph: launch each run's whole
    schedule as one CUDA graph (needs a non-default stream)."""
    c = mlmc_config()
    c.dim = w["dim"]
    c.n_levels = levels if levels is not None else w["levels"]
    for d in range(3):
        c.n0[d] = int(w["n0"][d]) if d < len(w["n0"]) else 1
        c.L[d] = float(w["L"][d]) if d < len(w["L"]) else 1.0
        c.stim_c[d] = float(w["stim_c"][d]) if d < len(w["stim_c"]) else 0.0
    c.m0 = w["m0"]
    c.T, c.c, c.a = w["T"], w["c"], w["a"]
    c.s_t, c.s_l0 = w["s_t"], w["s_l0"]
    c.theta0_deg, c.theta1_deg = w["theta0"], w["theta1"]
    c.stim_r = w["stim_r"]
    c.kl_sigma2, c.kl_ell, c.kl_modes = w["sigma2"], w["ell"], w["M"]
    c.precision = precision
    c.newton_tol, c.newton_max, c.lin_rtol, c.lin_max = newton_tol, newton_max, lin_rtol, lin_max
    c.solver = solver
    # the workload's own limit (key mixed_cdr_max) unless one is given
    c.mixed_cdr_max = float(w.get("mixed_cdr_max", 0.0) if mixed_cdr_max is None else mixed_cdr_max)
    c.cluster_size = cluster_size
    c.precond, c.mg_nu, c.mg_coarse_sweeps = precond, mg_nu, mg_coarse_sweeps
    c.use_graph = 1 if use_graph else 0
    # the paper's time scheme, applied-current pulse and final-state QoI (the
    # workload keys scheme / stim_kind / stim_amp / stim_sigma / stim_t1 / qoi)
    c.time_scheme = int(w.get("scheme", MLMC_SCHEME_IE))
    c.stim_kind = int(w.get("stim_kind", MLMC_STIM_BALL))
    c.stim_amp = float(w.get("stim_amp", 0.0))
    c.stim_sigma = float(w.get("stim_sigma", 1.0))
    c.stim_t1 = float(w.get("stim_t1", 0.0))
    c.qoi = int(w.get("qoi", MLMC_QOI_ACTIVATION))
    # the paper's KL variant (workload keys kl_kind / kl_tol / kl_s / kl_delta /
    # kl_cand_n; sigma2 and ell then describe the Gaussian covariance)
    c.kl_kind = int(w.get("kl_kind", MLMC_KL_SEPARABLE_EXP))
    c.kl_tol = float(w.get("kl_tol", 0.0))
    c.kl_s = float(w.get("kl_s", 0.3))
    c.kl_delta = float(w.get("kl_delta", 0.5))
    for d, v in enumerate(w.get("kl_cand_n", (0, 0, 0))):
        c.kl_cand_n[d] = int(v)
    return c


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Context:
    """One ``mlmc_ctx`` plus torch-allocated outputs and workspaces."""

    def __init__(self, cfg):
        self.cfg = cfg
        h = C.c_void_p()
        st = lib().mlmc_create(C.byref(cfg), C.byref(h))
        if st != MLMC_OK:
            raise MLMCError(st, lib().mlmc_last_error(None).decode())
        self.h = h
        self._ws = {}

    def close(self):
        if getattr(self, "h", None):
            lib().mlmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != MLMC_OK:
            raise MLMCError(st, lib().mlmc_last_error(self.h).decode())

    # ---------------------------------------------------------------- sizes
    def level_info(self, level):
        n, c, m = C.c_int64(), C.c_int64(), C.c_int32()
        self._check(lib().mlmc_level_info(self.h, level, C.byref(n), C.byref(c), C.byref(m)))
        return n.value, c.value, m.value

    def workspace_bytes(self, level, n):
        b = C.c_size_t()
        self._check(lib().mlmc_workspace_bytes(self.h, level, n, C.byref(b)))
        return b.value

    def run_workspace_bytes(self, N_l, batch):
        b = C.c_size_t()
        Nh = np.ascontiguousarray(N_l, np.int64)
        self._check(lib().mlmc_run_workspace_bytes(self.h, Nh.ctypes.data_as(C.c_void_p), batch,
                                                   C.byref(b)))
        return b.value

    def workspace(self, nbytes, key="ws"):
        import torch
        w = self._ws.get(key)
        if w is None or w.numel() < nbytes:
            w = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
            self._ws[key] = w
        return w

    # ---------------------------------------------------------------- steps
    def xi(self, seed, level, ids, stream=None):
        import torch
        ids = ids.to(device="cuda", dtype=torch.int64).contiguous()
        out = torch.empty((ids.numel(), self.cfg.kl_modes), dtype=torch.float64, device="cuda")
        self._check(lib().mlmc_xi(self.h, seed, level, _p(ids), ids.numel(), _p(out), _stream(stream)))
        return out

    def kl_field(self, level, xi, stream=None):
        import torch
        _, cells, _ = self.level_info(level)
        xi = xi.contiguous()
        out = torch.empty((xi.shape[0], cells), dtype=torch.float64, device="cuda")
        self._check(lib().mlmc_kl_field(self.h, level, _p(xi), xi.shape[0], _p(out), _stream(stream)))
        return out

    def kl_field_tc(self, level, xi, stream=None):
        """The field of kl_field on the tensor cores (split TF32, FP32 accuracy)."""
        import torch
        _, cells, _ = self.level_info(level)
        xi = xi.contiguous()
        n = xi.shape[0]
        out = torch.empty((n, cells), dtype=torch.float64, device="cuda")
        b = C.c_size_t()
        self._check(lib().mlmc_kl_tc_workspace_bytes(self.h, n, C.byref(b)))
        ws = self.workspace(max(b.value, 256), key="kl_tc")
        self._check(lib().mlmc_kl_field_tc(self.h, level, _p(xi), n, _p(out), _p(ws), ws.numel(),
                                           _stream(stream)))
        return out

    def solve(self, level, Z, slab=False, stream=None):
        import torch
        nodes, _, m = self.level_info(level)
        n = Z.shape[0]
        Z = Z.contiguous()
        t = torch.empty((n, nodes), dtype=torch.float64, device="cuda")
        sl = torch.empty((n, m + 1, nodes), dtype=torch.float64, device="cuda") if slab else None
        info = torch.zeros((n, 8), dtype=torch.int32, device="cuda")
        nb = self.workspace_bytes(level, n)
        ws = self.workspace(nb)
        self._check(lib().mlmc_solve(self.h, level, _p(Z), n, _p(t), _p(sl), _p(info), _p(ws),
                                     ws.numel(), _stream(stream)))
        return t, sl, info

    def slab_residual(self, level, Z, slab, full=True, stream=None):
        import torch
        n = slab.shape[0]
        nodes, _, m = self.level_info(level)
        F = torch.empty((n, m, nodes), dtype=torch.float64, device="cuda") if full else None
        rmax = torch.empty(n, dtype=torch.float64, device="cuda")
        self._check(lib().mlmc_slab_residual(self.h, level, _p(Z.contiguous()), _p(slab.contiguous()),
                                             n, _p(F), _p(rmax), _stream(stream)))
        return F, rmax

    def activation(self, level, slab, stream=None):
        import torch
        n = slab.shape[0]
        nodes, _, _ = self.level_info(level)
        t = torch.empty((n, nodes), dtype=torch.float64, device="cuda")
        self._check(lib().mlmc_activation(self.h, level, _p(slab.contiguous()), n, _p(t), _stream(stream)))
        return t

    def sample_level(self, level, seed, ids, want_maps=False, stream=None):
        import torch
        ids = ids.to(device="cuda", dtype=torch.int64).contiguous()
        n = ids.numel()
        n0, _, _ = self.level_info(0)
        y = torch.empty((n, n0), dtype=torch.float64, device="cuda")
        y2 = torch.empty_like(y)
        tf = tc = None
        if want_maps:
            tf = torch.empty((n, self.level_info(level)[0]), dtype=torch.float64, device="cuda")
            if level > 0:
                tc = torch.empty((n, self.level_info(level - 1)[0]), dtype=torch.float64, device="cuda")
        info = torch.zeros((2 * n, 8), dtype=torch.int32, device="cuda")
        nb = self.workspace_bytes(level, n)
        ws = self.workspace(nb)
        self._check(lib().mlmc_sample_level(self.h, level, seed, _p(ids), n, _p(y), _p(y2), _p(tf),
                                            _p(tc), _p(info), _p(ws), ws.numel(), _stream(stream)))
        return y, y2, tf, tc, info

    def accumulate(self, level, y, y2, stream=None):
        self._check(lib().mlmc_accumulate(self.h, level, _p(y.contiguous()), _p(y2.contiguous()),
                                          y.shape[0], _stream(stream)))

    def reset(self, stream=None):
        self._check(lib().mlmc_reset(self.h, _stream(stream)))

    def estimate(self, stream=None):
        L = self.cfg.n_levels
        n0, _, _ = self.level_info(0)
        mean, var = np.zeros(n0), np.zeros(n0)
        mean_l, var_l = np.zeros((L, n0)), np.zeros((L, n0))
        V = np.zeros(L)
        N = np.zeros(L, np.int64)
        rmse = C.c_double()
        dp = lambda a: a.ctypes.data_as(C.c_void_p)
        self._check(lib().mlmc_estimate(self.h, dp(mean), dp(var), dp(mean_l), dp(var_l), dp(V),
                                        dp(N), C.byref(rmse), _stream(stream)))
        return dict(mean=mean, var=var, mean_l=mean_l, var_l=var_l, V_l=V, N_l=N, rmse=rmse.value)

    def run(self, N_l, seed=0, batch=None, stream=None):
        """Whole MLMC run with fixed counts; host outputs (the end-to-end call).
        ``stats``: solve-kernel device ms, solve launches, CG and Newton
        node-iterations, truncations, halvings, failed solves, kernel launches."""
        L = self.cfg.n_levels
        batch = batch or int(max(N_l))
        n0, _, _ = self.level_info(0)
        Nh = np.ascontiguousarray(N_l, np.int64)
        mean, var, V, Cl = np.zeros(n0), np.zeros(n0), np.zeros(L), np.zeros(L)
        stats = np.zeros(9)
        rmse = C.c_double()
        nb = self.run_workspace_bytes(Nh, batch)
        ws = self.workspace(nb, key="run")
        dp = lambda a: a.ctypes.data_as(C.c_void_p)
        self._check(lib().mlmc_run(self.h, dp(Nh), seed, batch, _p(ws), ws.numel(), dp(mean), dp(var),
                                   dp(V), dp(Cl), C.byref(rmse), dp(stats), _stream(stream)))
        keys = ("solve_ms", "solve_launches", "cg_node_iters", "newton_node_iters", "truncations",
                "halvings", "failed", "launches", "cg64_node_iters")
        return dict(mean=mean, var=var, V_l=V, C_l=Cl, rmse=rmse.value, N_l=Nh,
                    stats=dict(zip(keys, stats.tolist())))

    def run_more(self, first_id, count, seed=0, batch=None, stream=None):
        """Adds pairs with ids first_id[l] .. first_id[l]+count[l]-1 per level to
        the running estimates (no reset).  Returns each level's solve seconds."""
        L = self.cfg.n_levels
        F = np.ascontiguousarray(first_id, np.int64)
        Nc = np.ascontiguousarray(count, np.int64)
        batch = batch or int(max(1, Nc.max()))
        secs = np.zeros(L)
        nb = self.run_workspace_bytes(Nc, batch)
        ws = self.workspace(nb, key="run")
        self._check(lib().mlmc_run_more(self.h, _dp(F), _dp(Nc), seed, batch, _p(ws), ws.numel(),
                                        _dp(secs), _stream(stream)))
        return secs

    def run_to_rmse(self, eps, N_pilot, max_rounds=8, max_per_level=1 << 20, seed=0, batch=64,
                    stream=None):
        """Adaptive MLMC to sampling error eps / sqrt(2) (mlmc_run_to_rmse).
        ``reached`` is False when the bias estimate exceeds eps / sqrt(2)
        (MLMC_WARN_BIAS: the RMSE target is out of reach of this hierarchy)."""
        L = self.cfg.n_levels
        n0, _, _ = self.level_info(0)
        P = np.ascontiguousarray(N_pilot, np.int64)
        N = np.zeros(L, np.int64)
        mean, var, V, Cl = np.zeros(n0), np.zeros(n0), np.zeros(L), np.zeros(L)
        rmse, bias = C.c_double(), C.c_double()
        nb = self.run_workspace_bytes(np.full(L, batch, np.int64), batch)
        ws = self.workspace(nb, key="run")
        st = lib().mlmc_run_to_rmse(self.h, eps, _dp(P), max_rounds, max_per_level, seed, batch,
                                    _p(ws), ws.numel(), _dp(N), _dp(mean), _dp(var), _dp(V),
                                    _dp(Cl), C.byref(rmse), C.byref(bias), _stream(stream))
        if st != MLMC_WARN_BIAS:
            self._check(st)
        return dict(N_l=N, mean=mean, var=var, V_l=V, C_l=Cl, rmse=rmse.value, bias=bias.value,
                    reached=st == MLMC_OK,
                    message=lib().mlmc_last_error(self.h).decode() if st != MLMC_OK else "")

    def kl_info(self):
        """(rank of the KL expansion, s_eff) (mlmc_kl_info)."""
        r, sv = C.c_int(), C.c_double()
        self._check(lib().mlmc_kl_info(self.h, C.byref(r), C.byref(sv)))
        return r.value, sv.value

    def check_timeout_path(self, polls):
        """polls >= 0: the tensor-core KL tiles time out on purpose (before
        issuing any work) and the group-layout solves' first barrier waits for
        one CTA too many (every sample reports MLMC_ERR_TIMEOUT); -1: normal
        operation (mlmc_check_timeout_path)."""
        self._check(lib().mlmc_check_timeout_path(self.h, int(polls)))

    def level_stats(self):
        """Per-level solve statistics (mlmc_level_stats): a list of dicts."""
        L = self.cfg.n_levels
        out = np.zeros(8 * L)
        self._check(lib().mlmc_level_stats(self.h, _dp(out)))
        keys = ("solve_ms", "solve_launches", "cg_node_iters", "newton_node_iters",
                "cg64_node_iters", "truncations", "halvings", "not_converged")
        return [dict(zip(keys, out[8 * l:8 * l + 8].tolist())) for l in range(L)]

    def diagnostics(self, stream=None):
        """Per-level ||mean(Y_l)||_w, the fitted weak rate alpha and the censored
        fractions of the running estimates (mlmc_diagnostics)."""
        L = self.cfg.n_levels
        nrm, cens = np.zeros(L), np.zeros(L)
        alpha = C.c_double()
        self._check(lib().mlmc_diagnostics(self.h, _dp(nrm), C.byref(alpha), _dp(cens),
                                           _stream(stream)))
        return dict(mean_norm=nrm, alpha=alpha.value, censored=cens)

    def autotune(self, level, n, seed=0, first_id=0, stream=None):
        """Times every feasible solve layout of ``level`` on n samples and keeps
        the fastest; returns (layout, {layout: ms})."""
        import torch
        ids = torch.arange(first_id, first_id + n, dtype=torch.int64, device="cuda")
        ws = self.workspace(self.workspace_bytes(level, n), key="tune")
        best = C.c_int()
        ms = np.zeros(16, np.float32)
        self._check(lib().mlmc_autotune(self.h, level, seed, _p(ids), n, _p(ws), ws.numel(),
                                        C.byref(best), _dp(ms), _stream(stream)))
        names = (-1, 1, 2, 4, 8, 16, 101, 102, 104, 108, 116, 301, 302, 304, 308,
                 MLMC_LAYOUT_GROUP)
        return best.value, {k: float(v) for k, v in zip(names, ms) if v >= 0}

    def layout(self, level):
        c = C.c_int()
        self._check(lib().mlmc_get_layout(self.h, level, C.byref(c)))
        return c.value

    def set_layout(self, level, layout):
        self._check(lib().mlmc_set_layout(self.h, level, layout))

    def get_state(self, stream=None):
        L = self.cfg.n_levels
        n0, _, _ = self.level_info(0)
        s = State.empty(L, n0)
        self._check(lib().mlmc_get_state(self.h, _dp(s.N), _dp(s.mean), _dp(s.m2), _dp(s.mean2),
                                         _stream(stream)))
        return s

    def set_state(self, s, stream=None):
        self._check(lib().mlmc_set_state(self.h, _dp(s.N), _dp(s.mean), _dp(s.m2), _dp(s.mean2),
                                         _stream(stream)))


class Server:
    """A request server on one Context (mlmc_server_*): submit level-pair
    requests at any time, poll finished results, read the running estimate.
    The Context must not be used directly while the server exists."""

    def __init__(self, ctx, max_batch=32, slots=4, mem_budget=1 << 30, keep_maps=False,
                 max_wait_s=0.0):
        self.ctx = ctx
        self.cfg = mlmc_server_config(max_batch, slots, mem_budget, int(keep_maps), max_wait_s)
        h = C.c_void_p()
        st = lib().mlmc_server_create(ctx.h, C.byref(self.cfg), C.byref(h))
        if st != MLMC_OK:
            raise MLMCError(st, lib().mlmc_last_error(ctx.h).decode())
        self.h = h
        self.n0 = ctx.level_info(0)[0]
        self.nL = ctx.level_info(ctx.cfg.n_levels - 1)[0]

    def close(self):
        if getattr(self, "h", None):
            lib().mlmc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != MLMC_OK:
            raise MLMCError(st, lib().mlmc_server_error(self.h).decode())

    @staticmethod
    def requests(tags, levels, seeds, sample_ids, stim=None):
        """A ctypes array of requests; stim [n][2 or 3] or None (configured centre)."""
        n = len(tags)
        arr = (mlmc_request * n)()
        for i in range(n):
            r = arr[i]
            r.tag, r.level, r.seed, r.sample_id = int(tags[i]), int(levels[i]), int(seeds[i]), \
                int(sample_ids[i])
            if stim is None:
                r.stim_c[0], r.stim_c[1], r.stim_c[2] = float("nan"), 0.0, 0.0
            else:
                c = list(stim[i]) + [0.0] * (3 - len(stim[i]))
                r.stim_c[0], r.stim_c[1], r.stim_c[2] = c[0], c[1], c[2]
        return arr

    def submit(self, reqs):
        self._check(lib().mlmc_server_submit(self.h, C.cast(reqs, C.c_void_p), len(reqs)))

    def poll(self, max_results=4096, timeout=0.0, want_y=False, want_maps=False):
        """Finished results as a list of dicts (with 'y' / 'map' arrays if asked)."""
        out = (mlmc_result * max_results)()
        cnt = C.c_int()
        y = np.zeros((max_results, self.n0)) if want_y else None
        maps = np.zeros((max_results, self.nL)) if want_maps else None
        self._check(lib().mlmc_server_poll(self.h, C.cast(out, C.c_void_p), max_results, C.byref(cnt),
                                           None if y is None else _dp(y),
                                           None if maps is None else _dp(maps), self.nL, timeout))
        res = []
        for i in range(cnt.value):
            r = out[i]
            d = dict(tag=r.tag, level=r.level, status=r.status, newton_iters=r.newton_iters,
                     cg_iters=r.cg_iters, t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done)
            if y is not None:
                d["y"] = y[i].copy()
            if maps is not None:
                nl = self.ctx.level_info(r.level)[0]
                d["map"] = maps[i, :nl].copy()
            res.append(d)
        return res

    def drain(self, timeout=600.0):
        self._check(lib().mlmc_server_drain(self.h, timeout))

    def stats(self):
        a = np.zeros(8, np.int64)
        self._check(lib().mlmc_server_stats(self.h, _dp(a)))
        keys = ("submitted", "queued", "inflight", "completed", "batches", "max_queue",
                "arena_peak_bytes", "error")
        return dict(zip(keys, a.tolist()))

    def clock(self):
        t = C.c_double()
        self._check(lib().mlmc_server_clock(self.h, C.byref(t)))
        return t.value

    def estimate(self):
        L = self.ctx.cfg.n_levels
        mean, var, V = np.zeros(self.n0), np.zeros(self.n0), np.zeros(L)
        N = np.zeros(L, np.int64)
        rmse, bias = C.c_double(), C.c_double()
        self._check(lib().mlmc_server_estimate(self.h, _dp(mean), _dp(var), _dp(V), _dp(N),
                                               C.byref(rmse), C.byref(bias)))
        return dict(mean=mean, var=var, V_l=V, N_l=N, rmse=rmse.value, bias=bias.value)


def info_dicts(info):
    """Per-sample solver reports from an info tensor [n][8]."""
    a = info.cpu().numpy()
    return [dict(zip(INFO_FIELDS, row[:7].tolist())) for row in a]
