"""One space dimension on the GPU against the oracle (the 1D+1 setting of
Sec. 4.1): solves on every layout with the bistable reaction (implicit Euler,
the ball stimulus) and with the stochastic heat equation (Crank-Nicolson, the
applied current, the final-state QoI, the paper's affine KL); level pairs; a
short run of the controlled-convergence experiment and its rates' signs."""
import numpy as np
import pytest

import oracle as O
from helpers import affine_kl, oracle_field, oracle_level, oracle_levels
from paper_1911_06066_gb300 import binding as B
from paper_1911_06066_gb300 import experiments as E

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1911_06066_gb300 import build
    build.build()
    assert torch.cuda.is_available()


BISTABLE = dict(name="bistable1d", dim=1, L=(1.0,), n0=(40,), m0=16, levels=2, T=1.0,
                c=100.0, a=0.1, s_t=1e-3, s_l0=1e-3, theta0=0.0, theta1=0.0, stim_r=0.1,
                stim_c=(0.0, 0.0, 0.0), sigma2=0.04, ell=0.2, M=8, N=[4, 4], seed=0)


def layouts():
    return [("block", B.MLMC_SOLVER_BLOCK, 0), ("cluster", B.MLMC_SOLVER_CLUSTER, 0),
            ("gm1", B.MLMC_SOLVER_CLUSTER, 101), ("gm2", B.MLMC_SOLVER_CLUSTER, 102)]


@pytest.mark.parametrize("name,solver,code", layouts())
@pytest.mark.parametrize("w", [BISTABLE, E.HEAT1D_6LVL], ids=["bistable_ie", "heat_cn"])
def test_1d_solve_matches_oracle(w, name, solver, code):
    w = dict(w, levels=2)
    ctx = B.Context(B.make_config(w, solver=solver))
    if code:
        for l in range(2):
            ctx.set_layout(l, code)
    akl = affine_kl(w) if w.get("kl_kind", 0) == 1 else None
    for level in (0, 1):
        ids = [0, 5]
        Z = ctx.kl_field(level, ctx.xi(3, level, torch.tensor(ids)))
        q, slab, info = ctx.solve(level, Z, slab=True)
        torch.cuda.synchronize()
        lv = oracle_level(w, level)
        for r, i in enumerate(ids):
            assert B.info_dicts(info)[r]["status"] == 0
            Zo = oracle_field(w, level, 3, level, i, akl)
            assert np.abs(Z[r].cpu().numpy() - Zo).max() <= 1e-11 * max(1.0, np.abs(Zo).max())
            so, qo, _ = O.solve_sample(lv, Zo)
            assert np.abs(slab[r].cpu().numpy() - so).max() <= 1e-8
            assert np.abs(q[r].cpu().numpy() - qo).max() <= 1e-6 * w["T"]
    ctx.close()


def test_1d_level_pairs_match_oracle():
    w = dict(E.HEAT1D_6LVL, levels=3)
    akl = affine_kl(w)
    lv = oracle_levels(w)
    ctx = B.Context(B.make_config(w))
    y, y2, _, _, info = ctx.sample_level(2, 9, torch.tensor([0, 1, 2]))
    torch.cuda.synchronize()
    for r in range(3):
        yo, y2o = O.sample_pair_affine(lv[2], lv[1], lv[0], akl, 2, 9, r)
        assert np.abs(y[r].cpu().numpy() - yo).max() <= 1e-10
        assert np.abs(y2[r].cpu().numpy() - y2o).max() <= 1e-10


def test_controlled_convergence_short_run():
    out = E.controlled_convergence_1d(B, reps=2, n_ref=512, mc_levels=3, mlmc_levels=3)
    mc = [x["rmse"] for x in out["mc"]]
    ml = [x["rmse"] for x in out["mlmc"]]
    assert all(np.isfinite(mc)) and all(np.isfinite(ml))
    # the errors fall with the level (controlled: sampling and discretisation
    # errors of the same order)
    assert mc[-1] < mc[0] and ml[-1] < ml[0]
