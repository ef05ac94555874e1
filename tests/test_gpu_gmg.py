"""Row a7: the geometric-multigrid preconditioner of the Newton steps' CG,
through the C ABI, against the CPU oracle (which solves every Newton step to
1e-12 with its own Jacobi-preconditioned CG).  On levels whose step Hessians
are positive definite (c dt max r' < 1) the Newton direction does not depend
on the preconditioner, so the GMG-preconditioned sweep must reach the oracle's
slab within the FP64 tolerances (max |du| <= 1e-8, activation times within
1e-6 T), and within 1e-4 T with the V-cycle in FP32 (mixed precision).
Grids: several multigrid levels, ragged (odd) cell counts that stop the
coarsening on some axes, 2D and 3D, the automatic layout and global-memory
clusters of 2 and 16 CTAs."""
import numpy as np
import pytest

import oracle as O
from helpers import oracle_level, small_workload
from paper_1911_06066_gb300 import binding as B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GMG = B.MLMC_PRECOND_GMG


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1911_06066_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def cdr(w, level):
    """c dt max r' of a level (max r' = c((1+a)^2/3 - a))."""
    dt = w["T"] / (w["m0"] * 2 ** level)
    return dt * w["c"] * ((1 + w["a"]) ** 2 / 3 - w["a"])


def make_ctx(w, layout=None, precision=B.MLMC_PREC_FP64, **kw):
    ctx = B.Context(B.make_config(w, precision, solver=B.MLMC_SOLVER_CLUSTER, **kw))
    if layout is not None:
        for l in range(w["levels"]):
            ctx.set_layout(l, layout)
    return ctx


def gpu_solve(ctx, w, level, ids, seed=0):
    Z = ctx.kl_field(level, ctx.xi(seed, level, torch.tensor(ids)))
    t, slab, info = ctx.solve(level, Z, slab=True)
    torch.cuda.synchronize()
    return t.cpu().numpy(), slab.cpu().numpy(), B.info_dicts(info)


_ORACLE = {}


def oracle_solve(w, level, sid, seed=0):
    key = (id(w), level, sid, seed)
    if key not in _ORACLE:
        _ORACLE[key] = _oracle_solve(w, level, sid, seed)
    return _ORACLE[key]


def _oracle_solve(w, level, sid, seed):
    lv = oracle_level(w, level)
    xo = O.xi(seed, level, sid, w["M"])
    Zo = O.kl_field(w["dim"], w["L"], list(lv.n)[:w["dim"]], w["sigma2"], w["ell"], w["M"], xo)[0]
    so, to, _ = O.solve_sample(lv, Zo)
    return so, to


def check_against_oracle(w, level, ids, t, slab, infos, u_tol, t_tol):
    worst_u, worst_t = 0.0, 0.0
    for r, sid in enumerate(ids):
        assert infos[r]["status"] == 0, infos[r]
        so, to = oracle_solve(w, level, sid)
        amb = (np.abs(so - 0.5) < 1e-6).any(axis=0)
        assert amb.sum() <= 2
        if slab is not None:
            worst_u = max(worst_u, np.abs(slab[r] - so).max())
        worst_t = max(worst_t, np.abs(t[r] - to)[~amb].max())
    if u_tol is not None:
        assert worst_u <= u_tol, worst_u
    assert worst_t <= t_tol * w["T"], worst_t


# 3D slab, 32 x 32 x 8 cells (three multigrid levels: 33x33x9, 17x17x5, 9x9x3
# nodes), dt = 5/256: every step Hessian is positive definite.
W3 = small_workload(dim=3, n0=(32, 32, 8), m0=128, levels=1, M=32, ell=0.1, T=2.5)
# 2D, 64 x 64 cells (65^2, 33^2, 17^2 nodes), dt = 5/256.
W2 = small_workload(dim=2, n0=(64, 64), m0=128, levels=1, M=16, ell=0.2, T=2.5)
# Ragged 3D: 18 x 10 x 5 cells; z (odd) is never halved, x and y once.
WR = small_workload(dim=3, n0=(18, 10, 5), m0=64, levels=1, M=12, ell=0.1, T=1.25)


def test_workloads_are_in_the_positive_definite_regime():
    for w in (W3, W2, WR):
        assert cdr(w, 0) < 1.0


@pytest.mark.parametrize("w,layout", [(W3, None), (W3, 102), (W2, None), (W2, 116), (WR, None),
                                      (WR, 102)])
def test_gmg_fp64_matches_oracle(w, layout):
    ctx = make_ctx(w, layout, precond=GMG)
    assert ctx.layout(0) == (layout or 0)
    ids = [0, 3]
    t, slab, infos = gpu_solve(ctx, w, 0, ids)
    check_against_oracle(w, 0, ids, t, slab, infos, 1e-8, 1e-6)


@pytest.mark.parametrize("w", [W3, W2])
def test_gmg_mixed_matches_oracle(w):
    """The V-cycle and the CG in FP32 inside the FP64 Newton iteration."""
    ctx = make_ctx(w, precision=B.MLMC_PREC_MIXED, precond=GMG)
    ids = [0, 3]
    t, _, infos = gpu_solve(ctx, w, 0, ids)
    check_against_oracle(w, 0, ids, t, None, infos, None, 1e-4)


def test_gmg_and_jacobi_agree_and_gmg_needs_fewer_cg_iterations():
    """Diffusion-dominated steps (conductivities x 20, 48^2 x 12 cells):
    dt K dominates M, Jacobi-CG needs many iterations per Newton step and the
    V-cycle few; both reach the same slab."""
    w = small_workload(dim=3, n0=(48, 48, 12), m0=128, levels=1, M=16, ell=0.1, T=2.5,
                       s_t=5e-3, s_l0=2e-2)
    ids = [4, 5]
    tj, sj, ij = gpu_solve(make_ctx(w, 116), w, 0, ids)
    tg, sg, ig = gpu_solve(make_ctx(w, 116, precond=GMG), w, 0, ids)
    assert all(i["status"] == 0 for i in ij + ig)
    assert np.abs(sj - sg).max() <= 1e-9
    cg_j = sum(i["cg_iters"] for i in ij)
    cg_g = sum(i["cg_iters"] for i in ig)
    assert cg_g * 2 <= cg_j, (cg_g, cg_j)


@pytest.mark.parametrize("nu,coarse", [(1, 4), (3, 16)])
def test_gmg_smoothing_counts(nu, coarse):
    ctx = make_ctx(W2, precond=GMG, mg_nu=nu, mg_coarse_sweeps=coarse)
    ids = [3]
    t, slab, infos = gpu_solve(ctx, W2, 0, ids)
    check_against_oracle(W2, 0, ids, t, slab, infos, 1e-8, 1e-6)


def test_gmg_is_not_used_on_indefinite_levels():
    """Where c dt max r' >= 1 the level keeps Jacobi: the result is bitwise the
    one of the Jacobi configuration."""
    w = small_workload(dim=2, n0=(32, 32), m0=32, levels=1, M=16, ell=0.2)
    assert cdr(w, 0) >= 1.0
    ids = [0, 1]
    tj, sj, _ = gpu_solve(make_ctx(w, 104), w, 0, ids)
    tg, sg, _ = gpu_solve(make_ctx(w, 104, precond=GMG), w, 0, ids)
    assert np.array_equal(sj, sg) and np.array_equal(tj, tg)
