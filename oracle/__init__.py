"""Oracle for the space-time MLMC monodomain path (arXiv:1911.06066).

TEST INFRASTRUCTURE ONLY.  A plain, slow FP64 CPU implementation, written
from the paper, that the CUDA path is checked against.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the product package never does, and the two share no code.

The arithmetic lives in C (``rng.c``, ``kl.c``, ``fem.c``, ``solve.c``,
``mlmc.c``, built by ``build.py``); this module only marshals arguments and
composes the estimators of Sec. 3.1.2 (Eq. MC-estimator, Eq. MLMC-estimator).

Functions without an independent pin are listed as "parity unpinned" in
their docstrings (none at present).
"""
import ctypes as C
import concurrent.futures
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _declare(_lib)
    return _lib


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


class Level(C.Structure):
    """One discretisation level (mirrors ``or_level`` in oracle.h)."""
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("m", C.c_int),
                ("L", C.c_double * 3), ("T", C.c_double), ("c", C.c_double),
                ("a", C.c_double), ("s_t", C.c_double), ("s_l0", C.c_double),
                ("theta0", C.c_double), ("theta1", C.c_double), ("stim_r", C.c_double),
                ("stim_c", C.c_double * 3), ("newton_tol", C.c_double),
                ("newton_max", C.c_int), ("lin_rtol", C.c_double), ("lin_max", C.c_int),
                ("scheme", C.c_int), ("stim_kind", C.c_int), ("stim_amp", C.c_double),
                ("stim_sigma", C.c_double), ("stim_t1", C.c_double), ("qoi", C.c_int),
                ("cond_kind", C.c_int)]

    @property
    def nodes(self):
        return lib().or_nodes(C.byref(self))

    @property
    def cells(self):
        return lib().or_cells(C.byref(self))

    @property
    def dt(self):
        return self.T / self.m

    def shape_nodes(self):
        return tuple(self.n[d] + 1 for d in range(self.dim))[::-1]


def make_level(dim, n, m, L, T, c, a, s_t, s_l0, theta0, theta1=None, stim_r=0.1,
               stim_c=(0.0, 0.0, 0.0), newton_tol=1e-12, newton_max=5000,
               lin_rtol=1e-12, lin_max=5000, scheme=0, stim_kind=0, stim_amp=0.0,
               stim_sigma=1.0, stim_t1=0.0, qoi=0, cond_kind=0):
    """One discretisation level.  scheme: 0 implicit Euler, 1 Crank-Nicolson
    (Sec. 3.2); stim_kind: 0 the ball u0 = 1 (radius stim_r), 1 u0 = 0 and the
    applied current stim_amp exp(-|x - stim_c|^2 / stim_sigma^2) on [0, stim_t1)
    (Sec. 4 set-up); qoi: 0 activation time, 1 the final state u(T); cond_kind:
    0 the fiber tensor with s_l = s_l0 exp(Z), 1 the paper's isotropic
    G = s_l0 (1 + Z) (Sec. 3.1.1)."""
    lv = Level()
    lv.dim = dim
    for d in range(3):
        lv.n[d] = int(n[d]) if d < len(n) else 1
        lv.L[d] = float(L[d]) if d < len(L) else 1.0
        lv.stim_c[d] = float(stim_c[d]) if d < len(stim_c) else 0.0
    lv.m, lv.T, lv.c, lv.a = int(m), float(T), float(c), float(a)
    lv.s_t, lv.s_l0 = float(s_t), float(s_l0)
    lv.theta0 = float(theta0)
    lv.theta1 = float(theta0 if theta1 is None else theta1)
    lv.stim_r = float(stim_r)
    lv.newton_tol, lv.newton_max = float(newton_tol), int(newton_max)
    lv.lin_rtol, lv.lin_max = float(lin_rtol), int(lin_max)
    lv.scheme, lv.stim_kind, lv.qoi = int(scheme), int(stim_kind), int(qoi)
    lv.stim_amp, lv.stim_sigma, lv.stim_t1 = float(stim_amp), float(stim_sigma), float(stim_t1)
    lv.cond_kind = int(cond_kind)
    return lv


def _declare(l):
    u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
    lp = C.POINTER(Level)
    l.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
    l.or_log.argtypes = [C.c_double]
    l.or_log.restype = C.c_double
    l.or_sincos_2pi.argtypes = [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    l.or_xi.argtypes = [C.c_uint64, C.c_int, C.c_uint64, C.c_int, _dp]
    l.or_psi_uniform.argtypes = [C.c_uint64, C.c_int, C.c_uint64, C.c_int, _dp]
    l.or_pivoted_cholesky.argtypes = [C.c_int, C.c_int, _dp, C.c_double, C.c_double, C.c_int,
                                      C.c_double, _ip, _dp, C.c_void_p]
    l.or_pc_eval.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_int, C.c_int,
                             _dp, _dp]
    l.or_kl_1d.argtypes = [C.c_double, C.c_double, C.c_int, _dp, _dp, _dp]
    l.or_kl_phi_1d.argtypes = [C.c_double, C.c_int, C.c_double, C.c_double, C.c_double]
    l.or_kl_phi_1d.restype = C.c_double
    l.or_kl_table.argtypes = [C.c_int, _dp, C.c_double, C.c_double, C.c_int, _ip, _dp]
    l.or_kl_field.argtypes = [C.c_int, _dp, _ip, C.c_double, C.c_double, C.c_int, C.c_int,
                              _dp, _dp]
    l.or_nodes.argtypes = [lp]
    l.or_cells.argtypes = [lp]
    l.or_assemble.argtypes = [lp, _dp, _dp, _dp]
    l.or_stiff_apply.argtypes = [lp, _dp, _dp, _dp]
    l.or_initial.argtypes = [lp, _dp]
    l.or_step_residual.argtypes = [lp, _dp, _dp, _dp, _dp, C.c_int, _dp]
    l.or_stimulus_step.argtypes = [lp, C.c_int, _dp]
    l.or_newton_cg.argtypes = [C.c_int, _dp, _dp, lp, _dp, _dp, _dp, C.POINTER(C.c_int)]
    l.or_step_solve.argtypes = [lp, _dp, _dp, _dp, C.c_int, _dp, _ip]
    l.or_step_gradient_flow.argtypes = [lp, _dp, _dp, _dp, C.c_int, C.c_void_p, _dp, C.c_double,
                                        C.c_double, C.c_int, _ip]
    l.or_solve_sample.argtypes = [lp, _dp, C.c_void_p, _dp, _dp, _ip]
    l.or_slab_residual.argtypes = [lp, _dp, _dp, _dp, _dp]
    l.or_activation.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp]
    l.or_inject.argtypes = [lp, lp, _dp, _dp]
    l.or_sample_pair.argtypes = [lp, lp, lp, C.c_double, C.c_double, C.c_int, C.c_uint64,
                                 C.c_int, C.c_uint64, _dp, _dp, C.POINTER(C.c_int)]


# ---------------------------------------------------------------- generator
def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al. 2011) -> 4 uint32."""
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def ln(x):
    return lib().or_log(float(x))


def sincos_2pi(u):
    s, c = C.c_double(), C.c_double()
    lib().or_sincos_2pi(float(u), C.byref(s), C.byref(c))
    return s.value, c.value


def xi(seed, level, sample_id, M):
    """Standard normals xi[0..M) of sample (seed, level pair, id)."""
    out = np.zeros(M, np.float64)
    lib().or_xi(int(seed), int(level), int(sample_id), int(M), out)
    return out


def xi_batch(seed, level, sample_ids, M):
    return np.stack([xi(seed, level, int(i), M) for i in sample_ids]) if len(sample_ids) \
        else np.zeros((0, M))


# ---------------------------------------------------------------- KL
def kl_1d(length, ell, n):
    om, lam, nrm = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().or_kl_1d(float(length), float(ell), int(n), om, lam, nrm)
    return om, lam, nrm


def kl_phi_1d(length, k, omega, nrm, x):
    return lib().or_kl_phi_1d(float(length), int(k), float(omega), float(nrm), float(x))


def kl_table(dim, L, sigma2, ell, M):
    idx = np.zeros(3 * M, np.int32)
    sl = np.zeros(M)
    rc = lib().or_kl_table(dim, np.asarray(list(L) + [1.0] * (3 - len(L)), np.float64),
                           float(sigma2), float(ell), int(M), idx, sl)
    if rc:
        raise RuntimeError("or_kl_table failed: %d" % rc)
    return idx.reshape(M, 3), sl


def kl_field(dim, L, n, sigma2, ell, M, xis):
    xis = np.ascontiguousarray(np.atleast_2d(xis), np.float64)
    ns = xis.shape[0]
    cells = int(np.prod(n[:dim]))
    Z = np.zeros(ns * cells)
    rc = lib().or_kl_field(dim, np.asarray(list(L) + [1.0] * (3 - len(L)), np.float64),
                           np.asarray(list(n) + [1] * (3 - len(n)), np.int32), float(sigma2),
                           float(ell), int(M), ns, xis.ravel(), Z)
    if rc:
        raise RuntimeError("or_kl_field failed: %d" % rc)
    return Z.reshape(ns, cells)


# ---------------------------------------------------------------- the paper's KL
def psi_uniform(seed, level, sample_id, M):
    """psi[0..M) ~ U(-1, 1) of sample (seed, level pair, id) (Sec. 3.1.1)."""
    out = np.zeros(M, np.float64)
    lib().or_psi_uniform(int(seed), int(level), int(sample_id), int(M), out)
    return out


def cell_centroids(dim, L, n):
    """Cell centroids [cells][dim], x fastest."""
    axes = [(np.arange(n[d]) + 0.5) * L[d] / n[d] for d in range(dim)]
    grid = np.meshgrid(*axes[::-1], indexing="ij")
    return np.ascontiguousarray(np.stack([g.ravel() for g in grid[::-1]], axis=1))


def pivoted_cholesky(X, sigma2, ell, M, tol=0.0, want_L=False):
    """Pivoted Cholesky of the Gaussian covariance on points X[n][dim]:
    (rank m, pivots[m], Lpiv[M][M], L[n][M] or None)."""
    X = np.ascontiguousarray(X, np.float64)
    n, dim = X.shape
    piv = np.zeros(M, np.int32)
    Lpiv = np.zeros(M * M)
    L = np.zeros(n * M) if want_L else None
    m = lib().or_pivoted_cholesky(dim, n, X.ravel(), float(sigma2), float(ell), int(M), float(tol),
                                  piv, Lpiv, None if L is None else L.ctypes.data)
    return m, piv[:m].copy(), Lpiv.reshape(M, M), (None if L is None else L.reshape(n, M))


def pc_eval(Y, Xp, sigma2, ell, M, m, Lpiv):
    """The factor's columns at points Y[ny][dim] (Nystrom extension): [ny][M]."""
    Y = np.ascontiguousarray(Y, np.float64)
    ny, dim = Y.shape
    Phi = np.zeros(ny * M)
    lib().or_pc_eval(dim, ny, Y.ravel(), np.ascontiguousarray(Xp, np.float64).ravel(), float(sigma2),
                     float(ell), int(M), int(m), np.ascontiguousarray(Lpiv, np.float64).ravel(), Phi)
    return Phi.reshape(ny, M)


class AffineKL:
    """The paper's KL variant on a level hierarchy (Sec. 3.1.1 and Sec. 4):
    Z(x, y) = sum_k l_k(x) y_k with l_k the pivoted-Cholesky columns of the
    Gaussian covariance, pivots chosen among the cell centroids of the
    candidate grid `cand_n`, extended to every level's centroids; G = G0 (1 +
    s_eff Z) with s_eff = min(s, delta / max_x sum_k |l_k(x)|), the max over the
    candidate centroids."""

    def __init__(self, dim, L, cand_n, level_ns, sigma2, ell, M, tol, s, delta):
        self.dim, self.L, self.M = dim, list(L), M
        X = cell_centroids(dim, L, cand_n)
        self.m, self.piv, self.Lpiv, Lc = pivoted_cholesky(X, sigma2, ell, M, tol, want_L=True)
        self.Xp = X[self.piv]
        self.Phi = [pc_eval(cell_centroids(dim, L, n), self.Xp, sigma2, ell, M, self.m, self.Lpiv)
                    for n in level_ns]
        # the sup over x of sum_k |l_k(x)|, taken on the candidate grid (shared
        # by every hierarchy that uses the same grid)
        bound = float(np.abs(Lc).sum(axis=1).max())
        self.s_eff = min(s, delta / bound)

    def field(self, level, psi):
        psi = np.atleast_2d(psi)
        return self.s_eff * (psi @ self.Phi[level].T)


# ---------------------------------------------------------------- FEM / solve
def assemble(lv, Z):
    n = lv.nodes
    mass = np.zeros(n)
    kst = np.zeros(n * 3 ** lv.dim)
    lib().or_assemble(C.byref(lv), np.ascontiguousarray(Z, np.float64), mass, kst)
    return mass, kst


def stiff_apply(lv, kst, v):
    y = np.zeros(lv.nodes)
    lib().or_stiff_apply(C.byref(lv), kst, np.ascontiguousarray(v, np.float64), y)
    return y


def initial(lv):
    u0 = np.zeros(lv.nodes)
    lib().or_initial(C.byref(lv), u0)
    return u0


def step_residual(lv, mass, kst, u, u_prev, k=1):
    F = np.zeros(lv.nodes)
    lib().or_step_residual(C.byref(lv), mass, kst, np.ascontiguousarray(u, np.float64),
                           np.ascontiguousarray(u_prev, np.float64), int(k), F)
    return F


def stimulus_step(lv, k):
    """The applied current averaged over step k at every node."""
    s = np.zeros(lv.nodes)
    lib().or_stimulus_step(C.byref(lv), int(k), s)
    return s


def newton_cg(lv, mass, kst, u_lin, F):
    """Newton direction d (Jacobi-PCG on H d = -F, truncated on negative curvature).
    Returns (d, cg_iterations, truncated)."""
    d = np.zeros(lv.nodes)
    tr = C.c_int(0)
    it = lib().or_newton_cg(lv.nodes, mass, kst, C.byref(lv), np.ascontiguousarray(u_lin, np.float64),
                            np.ascontiguousarray(F, np.float64), d, C.byref(tr))
    return d, it, bool(tr.value)


def step_solve(lv, mass, kst, u_prev, k=1):
    """Time step k from u_prev.  Returns (u, stats{newton, cg, truncations, halvings})."""
    u = np.zeros(lv.nodes)
    st = np.zeros(4, np.int32)
    rc = lib().or_step_solve(C.byref(lv), mass, kst, np.ascontiguousarray(u_prev, np.float64),
                             int(k), u, st)
    if rc < 0:
        raise RuntimeError("oracle step did not converge")
    return u, dict(zip(("newton", "cg", "truncations", "halvings"), st.tolist()))


def step_gradient_flow(lv, mass, kst, u_prev, tau=None, ftol=1e-12, max_pseudo=1000000, v0=None,
                       k=1):
    """Solver-independent root of one implicit-Euler step: the end point of the
    gradient flow M v' = -F(v) of the step energy started at u_prev (the local
    minimum in whose basin u_prev lies; started at v0 instead when given), by
    strictly convex implicit-Euler
    pseudo-steps of length tau (default 1 / (2 (max r' - 1/dt)), which keeps every
    pseudo-step strictly convex).  Returns (u, stats{pseudo, newton, cg})."""
    if tau is None:
        s = lv.c * ((1 + lv.a) ** 2 / 3 - lv.a) - lv.m / lv.T
        tau = 0.5 / s if s > 0 else 1.0
    u = np.zeros(lv.nodes)
    st = np.zeros(3, np.int32)
    v0c = None if v0 is None else np.ascontiguousarray(v0, np.float64)
    rc = lib().or_step_gradient_flow(C.byref(lv), mass, kst, np.ascontiguousarray(u_prev, np.float64),
                                     int(k), None if v0c is None else v0c.ctypes.data, u,
                                     float(tau), float(ftol), int(max_pseudo), st)
    if rc < 0:
        raise RuntimeError("gradient flow did not reach the tolerance: %s" % st.tolist())
    return u, dict(zip(("pseudo", "newton", "cg"), st.tolist()))


def solve_sample(lv, Z, u0=None):
    """Sequential implicit Euler + Newton from u0 (default: the stimulus).
    Returns (slab[m+1][nodes], t_act, newton iterations per step)."""
    n = lv.nodes
    u0c = None if u0 is None else np.ascontiguousarray(u0, np.float64)
    slab = np.zeros((lv.m + 1) * n)
    t = np.zeros(n)
    per = np.zeros(lv.m, np.int32)
    rc = lib().or_solve_sample(C.byref(lv), np.ascontiguousarray(Z, np.float64),
                               None if u0c is None else u0c.ctypes.data, slab, t, per)
    if rc < 0:
        raise RuntimeError("oracle Newton failed at step %d" % (-rc))
    return slab.reshape(lv.m + 1, n), t, per


def slab_residual(lv, mass, kst, slab):
    F = np.zeros(lv.m * lv.nodes)
    lib().or_slab_residual(C.byref(lv), mass, kst, np.ascontiguousarray(slab, np.float64).ravel(), F)
    return F.reshape(lv.m, lv.nodes)


def activation(nodes, m, dt, T, slab):
    t = np.zeros(nodes)
    lib().or_activation(int(nodes), int(m), float(dt), float(T),
                        np.ascontiguousarray(slab, np.float64).ravel(), t)
    return t


def inject(fine, l0, f):
    out = np.zeros(l0.nodes)
    lib().or_inject(C.byref(fine), C.byref(l0), np.ascontiguousarray(f, np.float64), out)
    return out


# ---------------------------------------------------------------- MLMC
def sample_pair(fine, coarse, l0, sigma2, ell, M, seed, level, sample_id):
    """(y, y2, newton_iters) of one level pair, on the coarsest grid."""
    n0 = l0.nodes
    y, y2 = np.zeros(n0), np.zeros(n0)
    it = C.c_int(0)
    rc = lib().or_sample_pair(C.byref(fine), C.byref(coarse) if coarse is not None else None,
                              C.byref(l0), float(sigma2), float(ell), int(M), int(seed),
                              int(level), int(sample_id), y, y2, C.byref(it))
    if rc < 0:
        raise RuntimeError("oracle sample pair (level %d, id %d) failed: %d" % (level, sample_id, rc))
    return y, y2, it.value


def sample_pair_affine(fine, coarse, l0, akl, level, seed, sample_id):
    """(y, y2) of one level pair with the paper's KL variant: psi uniform for
    (seed, level, id), the affine field on both grids (levels `level` and
    `level` - 1 of `akl`), both problems solved, QoIs injected."""
    psi = psi_uniform(seed, level, sample_id, akl.M)
    out = []
    for lv, l in ((fine, level), (coarse, level - 1)):
        if lv is None:
            out.append(np.zeros(l0.nodes))
            continue
        Z = akl.field(l, psi)[0]
        _, q, _ = solve_sample(lv, Z)
        out.append(inject(lv, l0, q))
    return out[0] - out[1], out[0] ** 2 - out[1] ** 2


def level_pairs(levels, l, sigma2, ell, M, seed, sample_ids, threads=1):
    """Y and Y2 rows for the given sample ids of level pair l (ctypes drops the GIL,
    so a thread pool runs the C solves in parallel)."""
    fine = levels[l]
    coarse = levels[l - 1] if l > 0 else None

    def one(i):
        y, y2, _ = sample_pair(fine, coarse, levels[0], sigma2, ell, M, seed, l, i)
        return y, y2

    ids = [int(i) for i in sample_ids]
    if threads > 1:
        with concurrent.futures.ThreadPoolExecutor(threads) as ex:
            res = list(ex.map(one, ids))
    else:
        res = [one(i) for i in ids]
    Y = np.stack([r[0] for r in res]) if res else np.zeros((0, levels[0].nodes))
    Y2 = np.stack([r[1] for r in res]) if res else np.zeros((0, levels[0].nodes))
    return Y, Y2


class Welford:
    """Per-node running mean and M2 (Welford 1962), one sample at a time, in C."""

    def __init__(self, n):
        self.mean = np.zeros(n)
        self.m2 = np.zeros(n)
        self._w = _WelfordC()
        self._w.n = 0
        self._w.mean = self.mean.ctypes.data_as(C.POINTER(C.c_double))
        self._w.m2 = self.m2.ctypes.data_as(C.POINTER(C.c_double))

    @property
    def n(self):
        return self._w.n

    def add(self, y):
        y = np.ascontiguousarray(y, np.float64)
        lib().or_welford_add(C.byref(self._w), y.size, y.ctypes.data_as(C.POINTER(C.c_double)))

    def var(self):
        return self.m2 / (self.n - 1) if self.n > 1 else np.zeros_like(self.m2)


class _WelfordC(C.Structure):
    _fields_ = [("n", C.c_long), ("mean", C.POINTER(C.c_double)), ("m2", C.POINTER(C.c_double))]


def mlmc_estimate(levels, sigma2, ell, M, seed, N, threads=1):
    """MLMC estimate (Eq. MLMC-estimator) of the mean activation map on the
    coarsest grid with N[l] pairs on level l; sample ids 0..N[l]-1.

    Returns dict: mean, var (second-moment telescoping minus mean^2, clipped at
    0), mean_l, var_l (per-level Var(Y_l)), V_l (L2(D)-weighted with the coarsest
    lumped mass), bias (||mean(Y_L)||), rmse (sqrt(sum V_l/N_l + bias^2)).
    """
    l0 = levels[0]
    w0, _ = assemble(l0, np.zeros(l0.cells))
    L = len(N)
    mean = np.zeros(l0.nodes)
    m2nd = np.zeros(l0.nodes)
    out = {"mean_l": [], "var_l": [], "V_l": [], "N_l": list(N)}
    for l in range(L):
        Y, Y2 = level_pairs(levels, l, sigma2, ell, M, seed, range(N[l]), threads)
        wy, wy2 = Welford(l0.nodes), Welford(l0.nodes)
        for r in range(Y.shape[0]):
            wy.add(Y[r])
            wy2.add(Y2[r])
        mean += wy.mean
        m2nd += wy2.mean
        out["mean_l"].append(wy.mean.copy())
        out["var_l"].append(wy.var())
        out["V_l"].append(float(np.sum(w0 * wy.var())))
    out["mean"] = mean
    out["var"] = np.maximum(m2nd - mean * mean, 0.0)
    bias = float(np.sqrt(np.sum(w0 * out["mean_l"][-1] ** 2))) if L > 1 else 0.0
    out["bias"] = bias
    out["rmse"] = float(np.sqrt(sum(v / n for v, n in zip(out["V_l"], N)) + bias * bias))
    return out


def cores():
    return os.cpu_count() or 1
