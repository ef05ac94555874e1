"""Host logic of the multi-device run: id sharding, the Chan merge of
accumulator states (C ABI, CPU only), the gloo all-gather exchange with
world size 2, failure of a rank before the exchange, and checkpoints."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle as O
from helpers import oracle_levels, small_workload
from paper_1911_06066_gb300 import binding as B
from paper_1911_06066_gb300 import distributed as D
import dist_workers


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _welford_state(Ys, Y2s):
    L = len(Ys)
    n0 = Ys[0].shape[1]
    st = B.State.empty(L, n0)
    for l in range(L):
        wy, wy2 = O.Welford(n0), O.Welford(n0)
        for r in range(Ys[l].shape[0]):
            wy.add(Ys[l][r])
            wy2.add(Y2s[l][r])
        st.N[l] = Ys[l].shape[0]
        st.mean[l], st.m2[l], st.mean2[l] = wy.mean, wy.m2, wy2.mean
    return st


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_shard_covers_every_id_once(world):
    N = [0, 1, 5, 64, 1001]
    for l, n in enumerate(N):
        seen = []
        for r in range(world):
            f, c = D.shard(N, r, world)
            seen.extend(range(f[l], f[l] + c[l]))
            assert c[l] in (n // world, n // world + 1)
        assert seen == list(range(n))


def test_merge_states_equals_one_pass():
    # two-pass definition on the union: mean, sum of squared deviations,
    # mean of Y2 -- against the C merge of two Welford states
    rng = np.random.default_rng(5)
    L, n0 = 3, 17
    Ys = [rng.normal(l, 1.0 + l, size=(n, n0)) for l, n in enumerate([40, 9, 2])]
    Y2s = [rng.normal(size=(Y.shape[0], n0)) for Y in Ys]
    cut = [13, 0, 2]
    a = _welford_state([Y[:c] for Y, c in zip(Ys, cut)], [Y[:c] for Y, c in zip(Y2s, cut)])
    b = _welford_state([Y[c:] for Y, c in zip(Ys, cut)], [Y[c:] for Y, c in zip(Y2s, cut)])
    a.merge(b)
    for l in range(L):
        Y = Ys[l]
        assert a.N[l] == Y.shape[0]
        np.testing.assert_allclose(a.mean[l], Y.mean(0), rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(a.m2[l], ((Y - Y.mean(0)) ** 2).sum(0), rtol=1e-12)
        np.testing.assert_allclose(a.mean2[l], Y2s[l].mean(0), rtol=1e-13, atol=1e-14)


def test_merge_states_rejects_bad_arguments():
    a, b = B.State.empty(2, 3), B.State.empty(2, 3)
    b.N[1] = -1
    with pytest.raises(B.MLMCError):
        a.merge(b)
    l = B.lib()
    assert l.mlmc_merge_states(0, 3, None, None, None, None, None, None, None, None) == -1


def test_state_flat_round_trip():
    rng = np.random.default_rng(1)
    s = B.State(np.array([3, 0, 12345678901]), rng.normal(size=(3, 5)), rng.random((3, 5)),
                rng.normal(size=(3, 5)))
    t = B.State.from_array(s.as_array(), 3, 5)
    for k in ("N", "mean", "m2", "mean2"):
        np.testing.assert_array_equal(getattr(s, k), getattr(t, k))


def test_checkpoint_round_trip(tmp_path):
    rng = np.random.default_rng(2)
    s = B.State(np.array([7, 2]), rng.normal(size=(2, 4)), rng.random((2, 4)), rng.normal(size=(2, 4)))
    p = str(tmp_path / "ck.npz")
    D.save_checkpoint(p, s, [7, 2], 2**63 + 5, meta={"workload": "small"})
    t, nxt, seed, meta = D.load_checkpoint(p)
    assert list(nxt) == [7, 2] and seed == 2**63 + 5 and meta == {"workload": "small"}
    for k in ("N", "mean", "m2", "mean2"):
        np.testing.assert_array_equal(getattr(s, k), getattr(t, k))


def test_gloo_world2_sharded_oracle_equals_single_process(tmp_path):
    """Two gloo ranks each take half the ids of every level, exchange their
    states in one all-gather and merge in rank order: both ranks end with the
    state of one process that ran all ids."""
    w = small_workload(n0=(6, 6), m0=8, levels=2, M=6)
    w["N"] = [5, 3]
    seed = 11
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=dist_workers.gloo_merge_worker,
                         args=(r, 2, port, w, seed, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    ref = dist_workers.oracle_shard_state(w, 0, 1, seed)
    outs = [np.load(str(tmp_path / ("rank%d.npz" % r))) for r in range(2)]
    for k in ("N", "mean", "m2", "mean2"):
        np.testing.assert_array_equal(outs[0][k], outs[1][k])
    np.testing.assert_array_equal(outs[0]["N"], ref.N)
    for k in ("mean", "m2", "mean2"):
        np.testing.assert_allclose(outs[0][k], getattr(ref, k), rtol=1e-12, atol=1e-12)
    # and the merged level means are the oracle's MLMC estimator
    est = O.mlmc_estimate(oracle_levels(w), w["sigma2"], w["ell"], w["M"], seed, w["N"])
    np.testing.assert_allclose(outs[0]["mean"].sum(0), est["mean"], rtol=1e-12, atol=1e-12)


def test_gloo_rank_failure_before_exchange_is_an_error(tmp_path):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=dist_workers.gloo_fail_worker, args=(r, 2, port, str(tmp_path)))
             for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert procs[1].exitcode != 0
    assert procs[0].exitcode == 0
    assert open(str(tmp_path / "rank0.txt")).read().startswith("error")
