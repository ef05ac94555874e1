"""The request server (continuous batching on one context): results equal
alone and in a mix, per-request stimulus centres and seeds against the
oracle, the running estimate against a fixed-count run, memory-based
admission under a tight budget, and an open-loop Poisson load."""
import math

import numpy as np
import pytest

import oracle as O
from helpers import oracle_level, small_workload
from paper_1911_06066_gb300 import binding as B
from paper_1911_06066_gb300 import serving as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1911_06066_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def workload():
    return small_workload(n0=(4, 4), m0=16, levels=2, M=8, stim_r=0.3, s_l0=0.02, s_t=0.005,
                          sigma2=0.25, T=1.5)


def ctx_for(w, precision=B.MLMC_PREC_FP64):
    return B.Context(B.make_config(w, precision))


def collect(srv, n, timeout=120.0):
    out = {}
    srv.drain(timeout)
    while len(out) < n:
        for r in srv.poll(want_y=True, want_maps=True, timeout=0.1):
            out[r["tag"]] = r
    return out


def test_result_is_the_same_alone_and_in_a_mix():
    w = workload()
    probe = dict(tag=1000, level=1, seed=3, id=5, stim=(0.05, 0.1, 0.0))
    srv = B.Server(ctx_for(w), max_batch=8, slots=3, keep_maps=True)
    srv.submit(B.Server.requests([probe["tag"]], [1], [probe["seed"]], [probe["id"]], [probe["stim"]]))
    alone = collect(srv, 1)[1000]
    srv.close()
    rng = np.random.default_rng(0)
    n = 40
    tags = list(range(n)) + [1000]
    levels = list(rng.integers(0, 2, n)) + [1]
    seeds = list(rng.integers(0, 1 << 40, n)) + [probe["seed"]]
    ids = list(rng.integers(0, 1000, n)) + [probe["id"]]
    stim = [tuple(rng.uniform(0, 0.2, 2)) for _ in range(n)] + [probe["stim"]]
    order = rng.permutation(n + 1)
    pick = lambda a: [a[i] for i in order]
    srv = B.Server(ctx_for(w), max_batch=8, slots=3, keep_maps=True)
    srv.submit(B.Server.requests(pick(tags), pick(levels), pick(seeds), pick(ids), pick(stim)))
    mix = collect(srv, n + 1)[1000]
    assert srv.stats()["batches"] > 1
    assert alone["status"] == 0 and mix["status"] == 0
    assert np.array_equal(alone["y"], mix["y"])
    assert np.array_equal(alone["map"], mix["map"])


def test_per_request_stimulus_and_seed_match_oracle():
    w = workload()
    srv = B.Server(ctx_for(w), max_batch=4, slots=2, keep_maps=True)
    reqs = [(0, 1, 11, 2, (0.0, 0.0)), (1, 1, 2 ** 40 + 3, 9, (0.15, 0.05)), (2, 0, 7, 1, (0.2, 0.2)),
            (3, 1, 7, 1, None)]
    stim = [r[4] if r[4] is not None else (float("nan"), 0.0) for r in reqs]
    srv.submit(B.Server.requests([r[0] for r in reqs], [r[1] for r in reqs], [r[2] for r in reqs],
                                 [r[3] for r in reqs], stim))
    got = collect(srv, len(reqs))
    for tag, level, seed, sid, sc in reqs:
        c = sc if sc is not None else w["stim_c"][:2]
        wl = dict(w, stim_c=(c[0], c[1], 0.0))
        lv = oracle_level(wl, level, newton_max=500)
        Zo = O.kl_field(w["dim"], w["L"], list(lv.n)[:w["dim"]], w["sigma2"], w["ell"], w["M"],
                        O.xi(seed, level, sid, w["M"]))[0]
        so, to, _ = O.solve_sample(lv, Zo)
        near = (np.abs(so - 0.5) < 1e-6).any(axis=0)
        r = got[tag]
        assert r["status"] == 0
        assert np.abs(r["map"] - to)[~near].max() <= 1e-6 * w["T"]


def test_running_estimate_equals_fixed_count_run():
    w = workload()
    N = [20, 9]
    ref = ctx_for(w).run(N, seed=4, batch=5)
    srv = B.Server(ctx_for(w), max_batch=6, slots=4)
    tags, levels, ids = [], [], []
    for l in range(2):
        for i in range(N[l]):
            tags.append(len(tags)); levels.append(l); ids.append(i)
    perm = np.random.default_rng(1).permutation(len(tags))
    srv.submit(B.Server.requests([tags[i] for i in perm], [levels[i] for i in perm],
                                 [4] * len(tags), [ids[i] for i in perm]))
    srv.drain(120)
    est = srv.estimate()
    assert list(est["N_l"]) == N
    np.testing.assert_allclose(est["mean"], ref["mean"], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(est["V_l"], ref["V_l"], rtol=1e-10)
    assert math.isclose(est["rmse"], ref["rmse"], rel_tol=1e-10)


def test_memory_based_admission_under_a_tight_budget():
    w = workload()
    ctx = ctx_for(w)
    one = max(ctx.workspace_bytes(l, 1) for l in range(2))
    budget = 3 * one
    srv = B.Server(ctx, max_batch=16, slots=8, mem_budget=budget)
    n = 24
    srv.submit(B.Server.requests(range(n), [i % 2 for i in range(n)], [1] * n, range(n)))
    got = collect(srv, n)
    st = srv.stats()
    assert st["completed"] == n and st["error"] == 0
    assert st["arena_peak_bytes"] <= budget
    assert st["batches"] >= 4          # batches were cut down to what fits
    assert all(r["status"] == 0 for r in got.values())
    with pytest.raises(B.MLMCError, match="WORKSPACE"):
        B.Server(ctx_for(w), mem_budget=one // 4)


def test_bad_request_level_is_rejected():
    srv = B.Server(ctx_for(workload()))
    with pytest.raises(B.MLMCError, match="ERR_ARG"):
        srv.submit(B.Server.requests([0], [2], [0], [0]))


def test_open_loop_poisson_load_completes_with_latencies():
    w = workload()
    srv = B.Server(ctx_for(w, B.MLMC_PREC_MIXED), max_batch=16, slots=4, max_wait_s=0.002)
    sched = S.poisson_schedule(2000.0, 300, [0.7, 0.3], rng_seed=3, per_request_seed=True,
                               stim_box=(0.0, 0.2))
    rep = S.run_open_loop(srv, sched, timeout=300)
    assert rep["completed"] == 300 and rep["failed"] == 0
    assert 0 < rep["p50_ms"] <= rep["p99_ms"]
    assert sum(rep["N_l"]) == 300
