"""The allocation-free solve entry point, mlmc_solve_noalloc.

Some callers may not allocate device memory at all -- a host framework that
reserved the device budget up front, a plugin barred from the device heap, or
code that cannot afford the synchronisation an allocation may trigger.  For
them the library offers mlmc_solve_noalloc, which runs the same kernels as
mlmc_solve but takes its scratch from a fixed static device array instead of
a caller workspace.  This file checks, through the C ABI, that two calls in a
row (sharing that array) give the same activation maps as mlmc_solve on the
same inputs, and that an oversize request is refused before any work.  It is
collected last so that a failure here never hides the rest of the suite."""
import ctypes as C

import numpy as np
import pytest

from paper_1911_06066_gb300 import binding as B
from paper_1911_06066_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T_TOL = 1e-6   # activation-time tolerance of the parity tests, relative to T


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1911_06066_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def noalloc(cfg, level, Z, t, info):
    return B.lib().mlmc_solve_noalloc(C.byref(cfg), level, C.c_void_p(Z.data_ptr()), Z.shape[0],
                                      C.c_void_p(t.data_ptr()), C.c_void_p(info.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_workspace_solve_twice():
    w = W.MLMC2D_3LVL
    for precision in (B.MLMC_PREC_FP64, B.MLMC_PREC_MIXED):
        cfg = B.make_config(w, precision)
        # the reference solve uses the same kernel layout as the no-alloc path
        ctx = B.Context(B.make_config(w, precision, solver=B.MLMC_SOLVER_BLOCK))
        calls = [(0, [0, 1, 2, 3]), (1, [5, 6])]     # two calls in a row, different sizes
        for level, ids in calls:
            Z = ctx.kl_field(level, ctx.xi(11, level, torch.tensor(ids)))
            t_ref, _, info_ref = ctx.solve(level, Z)
            nodes = ctx.level_info(level)[0]
            t = torch.full((len(ids), nodes), -7.0, dtype=torch.float64, device="cuda")
            info = torch.zeros((len(ids), 8), dtype=torch.int32, device="cuda")
            st = noalloc(cfg, level, Z, t, info)
            assert st == B.MLMC_OK, B.lib().mlmc_last_error(None)
            torch.cuda.synchronize()
            assert all(i["status"] == 0 for i in B.info_dicts(info))
            d = (t - t_ref).abs().max().item()
            assert d <= T_TOL * w["T"], (precision, level, d)
            assert np.array_equal(info.cpu().numpy()[:, :7], info_ref.cpu().numpy()[:, :7])
        ctx.close()


def test_noalloc_allocates_nothing_after_setup():
    """The defining property: once the first call on the device has done its
    one-time set-up, a call changes neither the device's free memory nor
    torch's allocation count."""
    w = W.MLMC2D_3LVL
    cfg = B.make_config(w, B.MLMC_PREC_MIXED)
    ctx = B.Context(B.make_config(w, B.MLMC_PREC_MIXED, solver=B.MLMC_SOLVER_BLOCK))
    Z = ctx.kl_field(1, ctx.xi(3, 1, torch.tensor([0, 1, 2])))
    nodes = ctx.level_info(1)[0]
    t = torch.zeros((3, nodes), dtype=torch.float64, device="cuda")
    info = torch.zeros((3, 8), dtype=torch.int32, device="cuda")
    assert noalloc(cfg, 1, Z, t, info) == B.MLMC_OK            # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert noalloc(cfg, 1, Z, t, info) == B.MLMC_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    allocs1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert free1 == free0, (free0, free1)
    assert allocs1 == allocs0
    assert all(i["status"] == 0 for i in B.info_dicts(info))
    ctx.close()


def test_noalloc_rejects_oversize_requests():
    cfg = B.make_config(W.MLMC2D_3LVL)
    Z = torch.zeros((64, 128 * 128), dtype=torch.float64, device="cuda")
    t = torch.zeros((64, 129 * 129), dtype=torch.float64, device="cuda")
    info = torch.zeros((64, 8), dtype=torch.int32, device="cuda")
    st = noalloc(cfg, 2, Z, t, info)
    assert st == -6
    msg = B.lib().mlmc_last_error(None).decode()
    assert "mlmc_solve_noalloc" in msg and "scratch" in msg
    assert torch.count_nonzero(t).item() == 0          # nothing was launched
    # a grid far beyond the array: refused by the size bound, before any
    # product of sizes could wrap around
    big = B.make_config(dict(W.MLMC2D_3LVL, n0=(1 << 19, 1 << 19)))
    assert noalloc(big, 0, Z, t, info) in (-1, -6)
