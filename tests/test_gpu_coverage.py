"""Configurations of the hot path checked at (or near) their full size:

* the 3D level 1 (64x64x16, c dt max r' = 2.37: several roots per step) against
  the oracle on the full grid for its first 4 steps (the oracle needs tens of
  minutes for all 64 steps at this size);
* the full-size 3D level 2 (128x128x32, 128 steps, FP32 inner solves in the
  mixed path) against the FP64 GPU solve, which is oracle-pinned;
* the 3-level 2D benchmark estimate (N_l = 512/128/32): the mixed-precision
  MLMC mean map within 0.1 eps of the FP64 one at every coarsest node;
* a request of the 2D 128^2 level served alone and inside a mix of other
  requests: bitwise the same result;
* the tensor-core KL field against the oracle's field directly."""
import numpy as np
import pytest

import oracle as O
from helpers import oracle_level
from paper_1911_06066_gb300 import binding as B
from paper_1911_06066_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1911_06066_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def test_slab3d_level1_full_grid_matches_oracle():
    steps = 4
    base = W.SLAB3D_4LVL
    m1 = base["m0"] * 2
    # the level's grid and time step, first `steps` steps: T scaled, m0 scaled
    w = dict(base, T=base["T"] * steps / m1, m0=steps // 2, levels=2)
    lv = oracle_level(w, 1)
    assert lv.n[0] == 64 and lv.n[2] == 16 and abs(lv.T / lv.m - base["T"] / m1) < 1e-15
    Zo = O.kl_field(3, w["L"], [64, 64, 16], w["sigma2"], w["ell"], w["M"], O.xi(0, 1, 3, w["M"]))[0]
    so, to, _ = O.solve_sample(lv, Zo)
    for precision in (B.MLMC_PREC_FP64, B.MLMC_PREC_MIXED):
        ctx = B.Context(B.make_config(w, precision))
        Z = ctx.kl_field(1, ctx.xi(0, 1, torch.tensor([3])))
        assert np.abs(Z[0].cpu().numpy() - Zo).max() <= 1e-13 * np.abs(Zo).max()
        t, slab, info = ctx.solve(1, Z, slab=True)
        torch.cuda.synchronize()
        assert B.info_dicts(info)[0]["status"] == 0
        # c dt max r' = 2.37 > 2: the mixed path keeps FP64 inner solves here,
        # so both precisions are held to the FP64 tolerances
        assert np.abs(slab[0].cpu().numpy() - so).max() <= 1e-8
        assert np.abs(t[0].cpu().numpy() - to).max() <= 1e-6 * base["T"]
        ctx.close()


def test_slab3d_level2_full_size_mixed_matches_fp64():
    w = W.SLAB3D_4LVL
    out = {}
    for precision in (B.MLMC_PREC_FP64, B.MLMC_PREC_MIXED):
        ctx = B.Context(B.make_config(w, precision))
        Z = ctx.kl_field(2, ctx.xi(0, 2, torch.tensor([1])))
        t, _, info = ctx.solve(2, Z)
        torch.cuda.synchronize()
        assert B.info_dicts(info)[0]["status"] == 0
        out[precision] = t[0].cpu().numpy()
        ctx.close()
    d = np.abs(out[B.MLMC_PREC_MIXED] - out[B.MLMC_PREC_FP64]).max()
    assert d <= 1e-4 * w["T"], d


def test_benchmark_estimate_mixed_mean_within_a_tenth_of_eps():
    w = W.MLMC2D_3LVL
    eps = 1e-3 * w["T"]
    means = {}
    for precision in (B.MLMC_PREC_FP64, B.MLMC_PREC_MIXED):
        ctx = B.Context(B.make_config(w, precision))
        means[precision] = ctx.run(w["N"], seed=1, batch=512)["mean"]
        ctx.close()
    d = np.abs(means[B.MLMC_PREC_MIXED] - means[B.MLMC_PREC_FP64]).max()
    assert d <= 0.1 * eps, d


def test_served_128_level_request_is_the_same_alone_and_in_a_mix():
    w = W.MLMC2D_3LVL
    probe = dict(tag=7000, level=2, seed=12345, id=9, stim=(0.15, 0.05, 0.0))

    def collect(srv, n):
        out = {}
        srv.drain(600.0)
        while len(out) < n:
            for r in srv.poll(want_y=True, want_maps=True, timeout=0.1):
                out[r["tag"]] = r
        return out

    ctx = B.Context(B.make_config(w, B.MLMC_PREC_MIXED))
    srv = B.Server(ctx, max_batch=16, slots=4, keep_maps=True, mem_budget=4 << 30)
    srv.submit(B.Server.requests([probe["tag"]], [2], [probe["seed"]], [probe["id"]], [probe["stim"]]))
    alone = collect(srv, 1)[7000]
    srv.close()
    rng = np.random.default_rng(1)
    n = 30
    tags = list(range(n)) + [7000]
    levels = list(rng.integers(0, 3, n)) + [2]
    seeds = list(rng.integers(0, 1 << 40, n)) + [probe["seed"]]
    ids = list(rng.integers(0, 1000, n)) + [probe["id"]]
    stim = [tuple(rng.uniform(0, 0.2, 2)) for _ in range(n)] + [probe["stim"]]
    order = rng.permutation(n + 1)
    pick = lambda a: [a[i] for i in order]
    srv = B.Server(ctx, max_batch=16, slots=4, keep_maps=True, mem_budget=4 << 30)
    srv.submit(B.Server.requests(pick(tags), pick(levels), pick(seeds), pick(ids), pick(stim)))
    mix = collect(srv, n + 1)[7000]
    assert srv.stats()["batches"] > 1
    srv.close()
    assert alone["status"] == 0 and mix["status"] == 0
    assert np.array_equal(alone["y"], mix["y"])
    assert np.array_equal(alone["map"], mix["map"])


@pytest.mark.parametrize("w,level,n", [(W.MLMC2D_3LVL, 1, 40), (W.SLAB3D_4LVL, 0, 33)])
def test_tc_field_matches_the_oracle_field(w, level, n):
    ctx = B.Context(B.make_config(w, B.MLMC_PREC_MIXED))
    ids = torch.arange(n)
    ztc = ctx.kl_field_tc(level, ctx.xi(5, level, ids)).cpu().numpy()
    lv = oracle_level(w, level)
    zo = O.kl_field(w["dim"], w["L"], list(lv.n)[:w["dim"]], w["sigma2"], w["ell"], w["M"],
                    np.stack([O.xi(5, level, int(i), w["M"]) for i in range(n)]))
    assert np.abs(ztc - zo).max() <= 4e-6 * np.abs(zo).max()
    ctx.close()
