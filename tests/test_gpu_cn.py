"""The paper's own discretisation on the GPU (Sec. 3.2 Crank-Nicolson blocks,
Sec. 3.3 reaction at the new time level, Sec. 4 applied-current pulse and the
final state as quantity of interest) against the oracle: every solve layout on
small 2D / 3D grids, the all-at-once slab residual, and the full-size levels 0
and 1 of the cube workload."""
import numpy as np
import pytest

import oracle as O
from helpers import oracle_field, oracle_level, small_workload
from paper_1911_06066_gb300 import binding as B
from paper_1911_06066_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAYOUTS = ["block", "cluster", "gm16", "gm2"]
CODE = {"gm16": 116, "gm2": 102}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1911_06066_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def cn_workload(dim, strong=False):
    """A shrunk problem with the paper's scheme and pulse; `strong`: a pulse
    large enough to start a front (activation-time QoI), else the literal
    sub-threshold pulse and the final-state QoI."""
    w = small_workload(dim=dim, n0=(6, 5) if dim == 2 else (4, 3, 3), m0=6, levels=2, M=8)
    w.update(scheme=B.MLMC_SCHEME_CN, stim_kind=B.MLMC_STIM_PULSE, stim_sigma=0.3,
             stim_c=(0.2, 0.3, 0.1), T=1.0, c=18.515, a=0.2435, s_t=3e-3, s_l0=5e-3,
             theta0=20.0, theta1=-40.0)
    if strong:
        w.update(stim_amp=30.0, stim_t1=0.12, qoi=B.MLMC_QOI_ACTIVATION)
    else:
        w.update(stim_amp=1.0, stim_t1=0.005, qoi=B.MLMC_QOI_FINAL_STATE)
    return w


def ctx_layout(w, layout, precision=B.MLMC_PREC_FP64):
    solver = B.MLMC_SOLVER_BLOCK if layout == "block" else B.MLMC_SOLVER_CLUSTER
    ctx = B.Context(B.make_config(w, precision, solver=solver))
    if layout in CODE:
        for l in range(w["levels"]):
            ctx.set_layout(l, CODE[layout])
    return ctx


def compare(w, level, ids, layout, precision=B.MLMC_PREC_FP64, u_tol=1e-8, q_tol=1e-8):
    ctx = ctx_layout(w, layout, precision)
    Z = ctx.kl_field(level, ctx.xi(0, level, torch.tensor(ids)))
    q, slab, info = ctx.solve(level, Z, slab=True)
    torch.cuda.synchronize()
    lv = oracle_level(w, level)
    for r, i in enumerate(ids):
        assert B.info_dicts(info)[r]["status"] == 0
        Zo = oracle_field(w, level, 0, level, i)
        assert np.abs(Z[r].cpu().numpy() - Zo).max() <= 1e-12 * max(1.0, np.abs(Zo).max())
        so, qo, _ = O.solve_sample(lv, Zo)
        assert np.abs(slab[r].cpu().numpy() - so).max() <= u_tol
        assert np.abs(q[r].cpu().numpy() - qo).max() <= q_tol
    ctx.close()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("dim", [2, 3])
def test_crank_nicolson_pulse_final_state(dim, layout):
    compare(cn_workload(dim), 1, [0, 3], layout)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_crank_nicolson_strong_pulse_activation(layout):
    w = cn_workload(2, strong=True)
    lv = oracle_level(w, 1)
    compare(w, 1, [1, 2], layout, q_tol=1e-6 * w["T"])


def test_crank_nicolson_slab_residual_matches_oracle():
    w = cn_workload(2, strong=True)
    ctx = B.Context(B.make_config(w))
    Z = ctx.kl_field(1, ctx.xi(0, 1, torch.tensor([4])))
    _, slab, _ = ctx.solve(1, Z, slab=True)
    F, rmax = ctx.slab_residual(1, Z, slab)
    torch.cuda.synchronize()
    lv = oracle_level(w, 1)
    mass, kst = O.assemble(lv, Z[0].cpu().numpy())
    Fo = O.slab_residual(lv, mass, kst, slab[0].cpu().numpy())
    assert np.abs(F[0].cpu().numpy().reshape(Fo.shape) - Fo).max() <= 1e-13 * mass.max() / lv.dt
    assert rmax[0].item() <= 1e-8


@pytest.mark.parametrize("level", [0, 1])
def test_cube_workload_full_size(level):
    w = W.CUBE_CN_4LVL
    compare(w, level, [0, 7], "cluster")
    compare(w, level, [5], "cluster", precision=B.MLMC_PREC_MIXED, u_tol=1e-4, q_tol=1e-4)
