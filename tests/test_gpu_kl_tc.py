"""Row a2 in the mixed-precision path: the KL synthesis on the tensor cores
(tcgen05, three-term split TF32 with FP32 accumulation) through the C ABI.

Checks: the field matches the FP64 synthesis (itself pinned to the oracle at
1e-13) to FP32 accuracy for 2D and 3D grids, 16 to 256 modes, batches that
fill one or several 32-sample tiles and ragged cell counts; a sample's field
does not depend on the batch it is computed in (bitwise); and a mixed-
precision solve driven by this field stays within 1e-4 T of the oracle's
activation times."""
import numpy as np
import pytest

import oracle as O
from helpers import oracle_level, small_workload
from paper_1911_06066_gb300 import binding as B
from paper_1911_06066_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1911_06066_gb300 import build
    build.build()
    assert torch.cuda.is_available()


CASES = [(W.MC2D_32, 0, 5), (W.MLMC2D_3LVL, 2, 33), (W.SLAB3D_4LVL, 1, 64),
         (W.SLAB3D_4LVL, 0, 300), (small_workload(n0=(5, 7), M=8), 1, 1),
         (small_workload(dim=3, n0=(3, 4, 2), M=40, ell=0.1), 1, 257)]


@pytest.mark.parametrize("w,level,n", CASES)
def test_tc_field_matches_fp64_synthesis(w, level, n):
    ctx = B.Context(B.make_config(w, B.MLMC_PREC_MIXED))
    xi = ctx.xi(11, level, torch.arange(n))
    z64 = ctx.kl_field(level, xi).cpu().numpy()
    ztc = ctx.kl_field_tc(level, xi).cpu().numpy()
    assert np.isfinite(ztc).all()
    scale = np.abs(z64).max()
    # FP32 operands and accumulation over M terms: a few FP32 ulps of the
    # largest partial sums
    assert np.abs(ztc - z64).max() <= 4e-6 * scale, np.abs(ztc - z64).max() / scale


def test_tc_field_does_not_depend_on_the_batch():
    w = W.MLMC2D_3LVL
    ctx = B.Context(B.make_config(w, B.MLMC_PREC_MIXED))
    ids = torch.arange(40, 140)
    xi = ctx.xi(3, 1, ids)
    full = ctx.kl_field_tc(1, xi).cpu().numpy()
    for lo, hi in [(0, 1), (17, 18), (5, 37), (64, 100)]:
        part = ctx.kl_field_tc(1, xi[lo:hi]).cpu().numpy()
        assert np.array_equal(part, full[lo:hi])


def test_tc_field_zero_and_error_cases():
    w = W.MC2D_32
    ctx = B.Context(B.make_config(w, B.MLMC_PREC_MIXED))
    xi = torch.zeros((3, w["M"]), dtype=torch.float64, device="cuda")
    assert np.array_equal(ctx.kl_field_tc(0, xi).cpu().numpy(), np.zeros((3, 32 * 32)))
    empty = ctx.kl_field_tc(0, xi[:0])
    assert empty.shape[0] == 0
    with pytest.raises(B.MLMCError):
        ctx.kl_field_tc(5, xi)


def test_mixed_solve_on_the_tc_field_matches_oracle():
    """2D 64^2 level of the 3-level workload (FP32 inner solves): the tensor-
    core field, the mixed sweep, activation within 1e-4 T of the FP64 oracle."""
    w = W.MLMC2D_3LVL
    level = 1
    ctx = B.Context(B.make_config(w, B.MLMC_PREC_MIXED))
    ids = [0, 9]
    Z = ctx.kl_field_tc(level, ctx.xi(0, level, torch.tensor(ids)))
    t, _, info = ctx.solve(level, Z)
    torch.cuda.synchronize()
    t = t.cpu().numpy()
    lv = oracle_level(w, level)
    for r, sid in enumerate(ids):
        assert B.info_dicts(info)[r]["status"] == 0
        xo = O.xi(0, level, sid, w["M"])
        Zo = O.kl_field(w["dim"], w["L"], list(lv.n)[:w["dim"]], w["sigma2"], w["ell"], w["M"], xo)[0]
        so, to, _ = O.solve_sample(lv, Zo)
        amb = (np.abs(so - 0.5) < 1e-6).any(axis=0)
        assert np.abs(t[r] - to)[~amb].max() <= 1e-4 * w["T"]


def test_bounded_wait_runs_out_and_is_reported():
    """The tensor-core kernel's bounded waits: with the check hook on, every
    tile waits on a barrier that nothing arms (before it issues any copy or
    MMA), gives up after a few polls and exits; the run reports
    MLMC_ERR_TIMEOUT and the context stays usable -- with the hook off, the
    next run equals one on a fresh context."""
    w = dict(W.MLMC2D_3LVL, levels=2)
    ctx = B.Context(B.make_config(w, B.MLMC_PREC_MIXED))
    ctx.check_timeout_path(1000)
    with pytest.raises(B.MLMCError) as e:
        ctx.run([4, 4], seed=3, batch=4)
    assert e.value.status == -4, str(e.value)
    ctx.check_timeout_path(-1)
    again = ctx.run([4, 4], seed=3, batch=4)
    fresh = B.Context(B.make_config(w, B.MLMC_PREC_MIXED)).run([4, 4], seed=3, batch=4)
    assert np.array_equal(again["mean"], fresh["mean"])
