"""Row a13: the CUDA-graph form of a run (mlmc_config.use_graph).  The whole
multi-stream schedule of one mlmc_run / mlmc_run_more call -- every batch of
every level, fine and coarse solves on their own streams -- is captured and
launched as one graph.  The estimate must be bitwise the one of the direct
launches; a second call with another seed updates the instantiated graph in
place, a call with other counts re-instantiates it, and the per-level solve
times (event nodes inside the graph) are still reported."""
import numpy as np
import pytest

from helpers import small_workload
from paper_1911_06066_gb300 import binding as B
from paper_1911_06066_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1911_06066_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def workload():
    return small_workload(n0=(8, 8), m0=16, levels=3, M=16, T=2.0)


def same(a, b):
    for k in ("mean", "var", "V_l"):
        assert np.array_equal(a[k], b[k]), k
    assert a["rmse"] == b["rmse"]
    assert a["stats"]["launches"] == b["stats"]["launches"]


@pytest.mark.parametrize("precision", [B.MLMC_PREC_FP64, B.MLMC_PREC_MIXED])
def test_graph_run_equals_direct_run(precision):
    w = workload()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        direct = B.Context(B.make_config(w, precision))
        graph = B.Context(B.make_config(w, precision, use_graph=True))
        for seed, N in [(1, [40, 12, 5]), (2, [40, 12, 5]), (3, [17, 30, 2]), (3, [17, 30, 2])]:
            a = direct.run(N, seed=seed, batch=16)
            b = graph.run(N, seed=seed, batch=16)
            same(a, b)
            assert np.all(b["C_l"] > 0)
    torch.cuda.synchronize()


def test_graph_run_more_and_legacy_stream():
    w = workload()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ref = B.Context(B.make_config(w))
        ref.reset()
        ref.run_more([0, 0, 0], [20, 6, 3], seed=5, batch=8)
        g = B.Context(B.make_config(w, use_graph=True))
        g.reset()
        secs = g.run_more([0, 0, 0], [20, 6, 3], seed=5, batch=8)
        assert np.all(secs > 0)
        ea, eb = ref.estimate(), g.estimate()
        assert np.array_equal(ea["mean"], eb["mean"]) and np.array_equal(ea["V_l"], eb["V_l"])
    # the legacy default stream cannot be captured: the call runs directly
    g2 = B.Context(B.make_config(w, use_graph=True))
    r = g2.run([20, 6, 3], seed=5, batch=8, stream=torch.cuda.default_stream())
    r0 = B.Context(B.make_config(w)).run([20, 6, 3], seed=5, batch=8,
                                          stream=torch.cuda.default_stream())
    same(r, r0)


def test_graph_benchmark_workload_batch():
    """One estimate of the 3-level 2D workload at reduced counts, as a graph."""
    w = W.MLMC2D_3LVL
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        a = B.Context(B.make_config(w, B.MLMC_PREC_MIXED)).run([64, 8, 2], seed=9, batch=64)
        b = B.Context(B.make_config(w, B.MLMC_PREC_MIXED, use_graph=True)).run([64, 8, 2], seed=9,
                                                                                batch=64)
    torch.cuda.synchronize()
    same(a, b)
