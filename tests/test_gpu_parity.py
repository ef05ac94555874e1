"""Parity of the CUDA path (through the C ABI) with the CPU oracle, row by row:
xi (bit-exact), the KL field, the per-sample Newton sweep (slab and activation
times), the all-at-once slab residual, activation extraction, level pairs and
the estimators.  Inputs are seeded and synthetic; each side draws its own xi.

Tolerances (FP64 path): max |du| <= 1e-8 over the slab and activation times
within 1e-6 T, except at nodes whose crossing is decided within 1e-6 of the
threshold 1/2 (the activation time is discontinuous there; those nodes are
counted and checked to be few).  Mixed path: activation within 1e-4 T."""
import math

import numpy as np
import pytest

import oracle as O
from helpers import oracle_level, oracle_levels, small_workload
from paper_1911_06066_gb300 import binding as B
from paper_1911_06066_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_TOL = 1e-8
T_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1911_06066_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def ctx_for(w, precision=B.MLMC_PREC_FP64, **kw):
    return B.Context(B.make_config(w, precision, **kw))


# solve layouts: the block-per-sample kernel, the automatic cluster layout
# (shared memory where a band fits), global-memory clusters of 16 and 2 CTAs,
# and global-memory clusters of 4 CTAs of 256 threads
LAYOUTS = [pytest.param("block", id="block"), pytest.param("cluster", id="cluster"),
           pytest.param("gm16", id="gm16"), pytest.param("gm2", id="gm2"),
           pytest.param("gm4x256", id="gm4x256")]
LAYOUT_CODE = {"gm16": 116, "gm2": 102, "gm4x256": 304}


def layout_ctx(w, layout, precision=B.MLMC_PREC_FP64, **kw):
    """A context whose every level uses the named layout."""
    solver = {"block": B.MLMC_SOLVER_BLOCK}.get(layout, B.MLMC_SOLVER_CLUSTER)
    if layout in (B.MLMC_SOLVER_AUTO, B.MLMC_SOLVER_BLOCK, B.MLMC_SOLVER_CLUSTER):
        solver = layout
    ctx = B.Context(B.make_config(w, precision, solver=solver, **kw))
    if layout in LAYOUT_CODE:
        for l in range(w["levels"]):
            ctx.set_layout(l, LAYOUT_CODE[layout])
    return ctx


def ambiguous_nodes(slab, thr=0.5, eps=1e-6):
    """Nodes whose activation decision lies within eps of the threshold."""
    near = np.abs(slab - thr) < eps
    return near.any(axis=0)


def compare_solve(w, level, sample_ids, seed=0, precision=B.MLMC_PREC_FP64, u_tol=U_TOL,
                  t_tol=T_TOL, solver=B.MLMC_SOLVER_AUTO):
    ctx = layout_ctx(w, solver, precision)
    ids = torch.tensor(sample_ids, dtype=torch.int64)
    xi = ctx.xi(seed, level, ids)
    Z = ctx.kl_field(level, xi)
    t, slab, info = ctx.solve(level, Z, slab=True)
    torch.cuda.synchronize()
    infos = B.info_dicts(info)
    lv = oracle_level(w, level)
    worst_u, worst_t, amb_total = 0.0, 0.0, 0
    for r, sid in enumerate(sample_ids):
        assert infos[r]["status"] == 0, infos[r]
        xo = O.xi(seed, level, sid, w["M"])
        Zo = O.kl_field(w["dim"], w["L"], list(lv.n)[:w["dim"]], w["sigma2"], w["ell"], w["M"], xo)[0]
        so, to, _ = O.solve_sample(lv, Zo)
        sg = slab[r].cpu().numpy()
        du = np.abs(sg - so).max()
        amb = ambiguous_nodes(so)
        dt_ = np.abs(t[r].cpu().numpy() - to)[~amb].max()
        worst_u, worst_t, amb_total = max(worst_u, du), max(worst_t, dt_), amb_total + amb.sum()
    assert worst_u <= u_tol, worst_u
    assert worst_t <= t_tol * w["T"], worst_t
    assert amb_total <= max(2, 0.001 * lv.nodes * len(sample_ids))
    return infos


# ------------------------------------------------------------------ row a1
@pytest.mark.parametrize("M", [1, 7, 16, 64, 256])
def test_xi_bit_exact(M):
    w = dict(W.MC2D_32, M=M)
    ctx = ctx_for(w)
    ids = [0, 1, 2, 3, 1000, 2 ** 32 + 5, 2 ** 40 + 123]
    for seed, level in [(0, 0), (12345, 2), (2 ** 33 + 7, 3)]:
        g = ctx.xi(seed, level, torch.tensor(ids)).cpu().numpy()
        o = np.stack([O.xi(seed, level, i, M) for i in ids])
        assert np.array_equal(g.view(np.uint64), o.view(np.uint64))


def test_xi_many_samples_bit_exact():
    ctx = ctx_for(dict(W.MLMC2D_3LVL))
    ids = np.arange(2000)
    g = ctx.xi(7, 1, torch.tensor(ids)).cpu().numpy()
    o = np.stack([O.xi(7, 1, int(i), 64) for i in ids])
    assert np.array_equal(g.view(np.uint64), o.view(np.uint64))


# ------------------------------------------------------------------ row a2
@pytest.mark.parametrize("w,level", [(W.MC2D_32, 0), (W.MLMC2D_3LVL, 2), (W.SLAB3D_4LVL, 1),
                                     (small_workload(n0=(5, 7), M=8), 1),
                                     (small_workload(dim=3, n0=(3, 4, 2), M=12, ell=0.1), 1)])
def test_kl_field(w, level):
    ctx = ctx_for(w)
    ids = [0, 5, 77]
    Z = ctx.kl_field(level, ctx.xi(3, level, torch.tensor(ids))).cpu().numpy()
    lv = oracle_level(w, level)
    Zo = O.kl_field(w["dim"], w["L"], list(lv.n)[:w["dim"]], w["sigma2"], w["ell"], w["M"],
                    np.stack([O.xi(3, level, i, w["M"]) for i in ids]))
    scale = np.abs(Zo).max()
    assert np.abs(Z - Zo).max() <= 1e-13 * scale + 1e-15


# ------------------------------------------------------------------ rows a3-a8
@pytest.mark.parametrize("solver", LAYOUTS)
def test_solve_mc2d_32_fp64(solver):
    """The plain-MC workload (32x32, 64 steps, 16 modes): several samples."""
    infos = compare_solve(W.MC2D_32, 0, [0, 1, 2, 15], solver=solver)
    assert max(i["truncations"] for i in infos) > 0      # the indefinite regime is exercised


@pytest.mark.parametrize("solver", LAYOUTS)
def test_solve_ragged_2d(solver):
    """24 x 38 nodes (ragged against the block sizes), dt = 0.1: c dt max r' = 3,
    so the step limit and negative-curvature truncation are exercised."""
    w = small_workload(n0=(23, 37), m0=20, levels=1, M=10, stim_r=0.35, T=2.0)
    compare_solve(w, 0, [0, 3, 4], solver=solver)


@pytest.mark.parametrize("solver", LAYOUTS)
def test_solve_ragged_3d(solver):
    w = small_workload(dim=3, n0=(6, 5, 3), m0=8, levels=1, M=12, ell=0.1, stim_r=0.35)
    compare_solve(w, 0, [1, 2], solver=solver)


@pytest.mark.parametrize("solver", LAYOUTS)
def test_solve_mlmc2d_level1_fp64(solver):
    """64^2 x 128 steps: two-CTA clusters (bands of 33 and 32 rows)."""
    compare_solve(W.MLMC2D_3LVL, 1, [0, 9], solver=solver)


@pytest.mark.parametrize("solver", LAYOUTS)
def test_solve_slab3d_level0_fp64(solver):
    """32x32x8 x 32 steps: 16-CTA clusters, bands of single z-planes, one empty."""
    compare_solve(W.SLAB3D_4LVL, 0, [0], solver=solver)


@pytest.mark.parametrize("solver", LAYOUTS)
def test_solve_mixed_spd_level_fp32_inner(solver):
    """Mixed precision at the finest 2D level (c dt max r' < 1): FP32 CG inside
    FP64 Newton converges to the same root."""
    compare_solve(W.MLMC2D_3LVL, 2, [4], precision=B.MLMC_PREC_MIXED, u_tol=1e-7, t_tol=1e-4,
                  solver=solver)


def test_mixed_keeps_fp64_inner_solves_on_strongly_indefinite_levels():
    """c dt max r' = 2.37 on the 32^2 level: with the default limit (2) the
    mixed configuration solves it with FP64 CG, so its results equal the FP64
    configuration's."""
    w = dict(W.MLMC2D_3LVL, mixed_cdr_max=0.0)
    outs = []
    for prec in (B.MLMC_PREC_FP64, B.MLMC_PREC_MIXED):
        ctx = ctx_for(w, prec)
        Z = ctx.kl_field(0, ctx.xi(0, 0, torch.arange(24)))
        t, _, info = ctx.solve(0, Z)
        outs.append((t.cpu().numpy(), info.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_fp32_inner_solves_on_the_benchmark_32_level_reach_the_fp64_roots():
    """The 2D benchmark workload raises the limit to 2.5: its 32^2 level
    (c dt max r' = 2.37, the gradient-flow continuation) runs FP32 CG inside
    the FP64 pseudo-steps and still ends every step in the FP64 root."""
    w = W.MLMC2D_3LVL
    outs = []
    for prec in (B.MLMC_PREC_FP64, B.MLMC_PREC_MIXED):
        ctx = ctx_for(w, prec)
        Z = ctx.kl_field(0, ctx.xi(0, 0, torch.arange(128)))
        t, _, info = ctx.solve(0, Z)
        assert all(d["status"] == 0 for d in B.info_dicts(info))
        outs.append(t.cpu().numpy())
    assert np.abs(outs[0] - outs[1]).max() <= 1e-6 * w["T"]


def test_cluster_and_block_layouts_agree_full_size():
    """128^2 x 256 steps, 8-CTA clusters vs one block per sample, FP64."""
    w = W.MLMC2D_3LVL
    res = []
    for solver in (B.MLMC_SOLVER_BLOCK, B.MLMC_SOLVER_CLUSTER):
        ctx = ctx_for(w, solver=solver)
        Z = ctx.kl_field(2, ctx.xi(5, 2, torch.tensor([0, 1])))
        t, _, info = ctx.solve(2, Z)
        res.append(t.cpu().numpy())
        assert all(i["status"] == 0 for i in B.info_dicts(info))
    assert np.abs(res[0] - res[1]).max() <= T_TOL * w["T"]


def test_slab_residual_matches_oracle():
    w = W.MC2D_32
    lv = oracle_level(w, 0)
    ctx = ctx_for(w)
    xo = O.xi(0, 0, 2, w["M"])
    Zo = O.kl_field(2, w["L"], [32, 32], w["sigma2"], w["ell"], w["M"], xo)[0]
    so, _, _ = O.solve_sample(lv, Zo)
    rng = np.random.default_rng(0)
    pert = so + 1e-3 * rng.standard_normal(so.shape)       # a non-converged slab too
    mass, kst = O.assemble(lv, Zo)
    for slab_np in (so, pert):
        F, rmax = ctx.slab_residual(0, torch.tensor(Zo[None]).cuda(), torch.tensor(slab_np[None]).cuda())
        Fo = O.slab_residual(lv, mass, kst, slab_np)
        scale = np.abs(mass).max() / lv.dt
        assert np.abs(F[0].cpu().numpy() - Fo).max() <= 1e-13 * scale
        assert math.isclose(rmax.item(), (np.abs(Fo) / mass).max(), rel_tol=1e-9, abs_tol=1e-14)


def test_activation_kernel_matches_oracle():
    rng = np.random.default_rng(1)
    w = small_workload(n0=(9, 6), m0=20, levels=1)
    lv = oracle_level(w, 0)
    slab = np.cumsum(rng.random((lv.m + 1, lv.nodes)) * 0.08, axis=0)
    slab[0, :3] = 0.7
    ctx = ctx_for(w)
    t = ctx.activation(0, torch.tensor(slab[None]).cuda())[0].cpu().numpy()
    to = O.activation(lv.nodes, lv.m, lv.dt, lv.T, slab)
    assert np.abs(t - to).max() <= 1e-14 * lv.T


def independent_step_checks(lv, Z, slab):
    """Rebuilt (3-point Gauss) residual of every step and the smallest
    eigenvalue of every step Hessian, for a slab produced by the CUDA path."""
    from test_oracle_solve import independent_operators
    mass, K = independent_operators(lv, Z)
    dt = lv.T / lv.m
    res, lam = 0.0, np.inf
    for k in range(1, lv.m + 1):
        u, up = slab[k], slab[k - 1]
        F = mass / dt * (u - up) + K @ u - mass * lv.c * u * (1 - u) * (u - lv.a)
        res = max(res, np.abs(F / mass).max())
        rp = lv.c * (-3 * u * u + 2 * (1 + lv.a) * u - lv.a)
        lam = min(lam, np.linalg.eigvalsh(K + np.diag(mass / dt - mass * rp)).min())
    return res, lam


@pytest.mark.parametrize("solver", LAYOUTS)
def test_strongly_indefinite_steps_give_valid_roots(solver):
    """c dt max r' = 5.7 (far stiffer than any workload level): which of the
    step's roots Newton reaches can depend on rounding, so the CUDA result is
    checked for what makes it a valid result of the method -- every step
    satisfies its residual and is a local minimum of its step energy."""
    w = small_workload(n0=(6, 6), m0=8, levels=1, M=8, stim_r=0.3, s_l0=0.02, s_t=0.005,
                       sigma2=0.25, T=1.5)
    ctx = layout_ctx(w, solver)
    ids = [0, 1, 5]
    Z = ctx.kl_field(0, ctx.xi(9, 0, torch.tensor(ids)))
    t, slab, info = ctx.solve(0, Z, slab=True)
    lv = oracle_level(w, 0)
    for r in range(len(ids)):
        assert B.info_dicts(info)[r]["status"] == 0
        res, lam = independent_step_checks(lv, Z[r].cpu().numpy(), slab[r].cpu().numpy())
        assert res < 1e-9 and lam > 0.0, (res, lam)


# ------------------------------------------------------------------ rows a9-a10
def test_sample_level_pairs():
    """Three levels with fronts that cross the coarse grids (c dt max r' = 1.9,
    0.95, 0.47: the regime of the workloads' finer levels)."""
    w = small_workload(n0=(6, 6), m0=24, levels=3, M=8, stim_r=0.3, s_l0=0.02, s_t=0.005,
                       sigma2=0.25, T=1.5)
    lvs = oracle_levels(w, newton_max=500)
    ctx = ctx_for(w, newton_max=500)
    ids = [0, 1, 5]
    for level in range(3):
        y, y2, tf, tc, info = ctx.sample_level(level, 9, torch.tensor(ids), want_maps=True)
        for r, sid in enumerate(ids):
            yo, y2o, _ = O.sample_pair(lvs[level], lvs[level - 1] if level else None, lvs[0],
                                       w["sigma2"], w["ell"], w["M"], 9, level, sid)
            assert np.abs(y[r].cpu().numpy() - yo).max() <= T_TOL * w["T"]
            assert np.abs(y2[r].cpu().numpy() - y2o).max() <= 2 * T_TOL * w["T"] ** 2


def test_accumulate_and_estimate():
    w = small_workload(n0=(4, 4), m0=8, levels=3, M=4)
    ctx = ctx_for(w)
    n0 = 25
    rng = np.random.default_rng(2)
    data = [[rng.normal(l, 1 + l, (nb, n0)) for nb in (7, 1, 12)] for l in range(3)]
    for l in range(3):
        for batch in data[l]:
            yy = torch.tensor(batch).cuda()
            ctx.accumulate(l, yy, yy * yy)
    est = ctx.estimate()
    w0, _ = O.assemble(oracle_level(w, 0), np.zeros(16))
    mean = np.zeros(n0); e2 = np.zeros(n0); r2 = 0.0
    for l in range(3):
        Y = np.concatenate(data[l])
        wf = O.Welford(n0)
        for row in Y:
            wf.add(row)
        np.testing.assert_allclose(est["mean_l"][l], wf.mean, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(est["var_l"][l], wf.var(), rtol=1e-11)
        assert est["N_l"][l] == len(Y)
        assert math.isclose(est["V_l"][l], float(np.sum(w0 * wf.var())), rel_tol=1e-11)
        mean += wf.mean
        e2 += np.mean(Y * Y, axis=0)
        r2 += est["V_l"][l] / len(Y)
    np.testing.assert_allclose(est["mean"], mean, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(est["var"], np.maximum(e2 - mean ** 2, 0), rtol=1e-9, atol=1e-10)
    bias = math.sqrt(np.sum(w0 * est["mean_l"][2] ** 2))
    assert math.isclose(est["rmse"], math.sqrt(r2 + bias ** 2), rel_tol=1e-12)


def test_run_matches_oracle_mlmc():
    w = small_workload(n0=(4, 4), m0=16, levels=2, M=8, stim_r=0.3, s_l0=0.02, s_t=0.005,
                       sigma2=0.25, T=1.5)
    lvs = oracle_levels(w, newton_max=500)
    ctx = ctx_for(w, newton_max=500)
    N = [24, 10]
    res = ctx.run(N, seed=1, batch=7)
    est = O.mlmc_estimate(lvs, w["sigma2"], w["ell"], w["M"], 1, N)
    np.testing.assert_allclose(res["mean"], est["mean"], atol=1e-6 * w["T"])
    np.testing.assert_allclose(res["V_l"], est["V_l"], rtol=1e-6, atol=1e-10)
    assert math.isclose(res["rmse"], est["rmse"], rel_tol=1e-6)
    assert np.all(res["C_l"] > 0)


# ------------------------------------------------------------------ edge cases
def test_empty_batches_and_errors():
    ctx = ctx_for(W.MC2D_32)
    e = torch.empty(0, dtype=torch.int64)
    assert ctx.xi(0, 0, e).shape == (0, 16)
    Z = torch.empty((0, 1024), dtype=torch.float64, device="cuda")
    t, _, _ = ctx.solve(0, Z)
    assert t.shape[0] == 0
    with pytest.raises(B.MLMCError, match="ERR_ARG"):
        ctx.kl_field(1, torch.zeros((1, 16), dtype=torch.float64, device="cuda"))
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    Z1 = torch.zeros((1, 1024), dtype=torch.float64, device="cuda")
    t1 = torch.zeros((1, 1089), dtype=torch.float64, device="cuda")
    import ctypes as C
    st = B.lib().mlmc_solve(ctx.h, 0, C.c_void_p(Z1.data_ptr()), 1, C.c_void_p(t1.data_ptr()), None,
                            None, C.c_void_p(ws.data_ptr()), 256, None)
    assert st == -6 and b"workspace" in B.lib().mlmc_last_error(ctx.h)


def test_non_convergence_is_reported_not_fatal():
    w = W.MC2D_32
    ctx = ctx_for(w, newton_max=2)
    xi = ctx.xi(0, 0, torch.arange(3))
    t, _, info = ctx.solve(0, ctx.kl_field(0, xi))
    infos = B.info_dicts(info)
    assert all(i["status"] == -3 and i["failed_step"] >= 1 for i in infos)
    # the context stays usable
    ctx2 = ctx_for(w)
    t2, _, info2 = ctx2.solve(0, ctx2.kl_field(0, ctx2.xi(0, 0, torch.arange(1))))
    assert B.info_dicts(info2)[0]["status"] == 0


def test_full_size_level2_pair_sampled():
    """The 3-level workload at full size: one level-2 pair (128^2 x 256 steps and
    64^2 x 128 steps) against the oracle."""
    w = W.MLMC2D_3LVL
    lvs = oracle_levels(w)
    ctx = ctx_for(w)
    y, y2, tf, tc, info = ctx.sample_level(2, 0, torch.tensor([3]), want_maps=True)
    yo, y2o, _ = O.sample_pair(lvs[2], lvs[1], lvs[0], w["sigma2"], w["ell"], w["M"], 0, 2, 3)
    assert all(i["status"] == 0 for i in B.info_dicts(info))
    d = np.abs(y[0].cpu().numpy() - yo)
    assert np.sort(d)[-3] <= T_TOL * w["T"]          # allow <= 2 threshold-ambiguous nodes


@pytest.mark.parametrize("precision", [B.MLMC_PREC_MIXED], ids=["mixed"])
def test_full_size_3d_level2_certified_by_the_slab_residual(precision):
    """The 3D slab's 128 x 128 x 32 level at full size (549,153 nodes, 128
    steps) in the benchmark's precision and automatic layout (global-memory
    clusters): too large for the oracle, so the solve is checked by what holds
    at any size -- the all-at-once residual of Eq. mono_disc over every slice
    vanishes to the Newton tolerance, the activation map recomputed from the
    stored slab equals the one extracted on the fly, and the front has moved."""
    w = W.SLAB3D_4LVL
    level = 2
    ctx = ctx_for(w, precision)
    Z = ctx.kl_field(level, ctx.xi(0, level, torch.tensor([5])))
    t, slab, info = ctx.solve(level, Z, slab=True)
    torch.cuda.synchronize()
    assert B.info_dicts(info)[0]["status"] == 0, B.info_dicts(info)
    _, rmax = ctx.slab_residual(level, Z, slab, full=False)
    # |F| / M_i <= (1/dt + |K_ii| / M_i) max|d| ~ 2e-10 for max|d| <= 1e-12
    assert rmax.item() <= 1e-8, rmax.item()
    t2 = ctx.activation(level, slab)
    assert torch.max(torch.abs(t - t2)).item() <= 1e-12 * w["T"]
    tn = t[0].cpu().numpy()
    assert (tn < w["T"]).sum() > 1000 and (tn == 0.0).sum() > 0
