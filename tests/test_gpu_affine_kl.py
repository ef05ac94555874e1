"""The paper's KL variant on the GPU (Sec. 3.1.1, Eq. KL-expansion-
deterministic; Sec. 4) against the oracle: the uniform inputs bit for bit,
the pivoted-Cholesky rank and the ellipticity-capped scale, the affine field
on every level in FP64 and on the tensor cores, and level pairs of the cube
workload (Crank-Nicolson, applied-current pulse, final-state QoI)."""
import numpy as np
import pytest

import oracle as O
from helpers import affine_kl, oracle_levels
from paper_1911_06066_gb300 import binding as B
from paper_1911_06066_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1911_06066_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def cube():
    return W.CUBE_CN_4LVL, affine_kl(W.CUBE_CN_4LVL)


def test_uniform_inputs_bit_exact(cube):
    w, _ = cube
    ctx = B.Context(B.make_config(w))
    ids = [0, 1, 17, 2 ** 33 + 9]
    for seed, level in [(0, 0), (991, 3)]:
        g = ctx.xi(seed, level, torch.tensor(ids)).cpu().numpy()
        o = np.stack([O.psi_uniform(seed, level, i, w["M"]) for i in ids])
        assert np.array_equal(g.view(np.uint64), o.view(np.uint64))


def test_rank_and_scale(cube):
    w, akl = cube
    ctx = B.Context(B.make_config(w))
    rank, s_eff = ctx.kl_info()
    assert rank == akl.m == 66
    assert abs(s_eff - akl.s_eff) <= 1e-12 * akl.s_eff


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_affine_field_fp64_and_tensor_cores(cube, level):
    w, akl = cube
    ctx = B.Context(B.make_config(w, B.MLMC_PREC_MIXED))
    n = 37
    xi = ctx.xi(4, level, torch.arange(n))
    z64 = ctx.kl_field(level, xi).cpu().numpy()
    ztc = ctx.kl_field_tc(level, xi).cpu().numpy()
    zo = np.stack([akl.field(level, O.psi_uniform(4, level, i, w["M"]))[0] for i in range(n)])
    scale = np.abs(zo).max()
    assert scale <= 0.5 + 1e-12                      # the ellipticity cap
    assert np.abs(z64 - zo).max() <= 1e-12 * scale
    assert np.abs(ztc - zo).max() <= 4e-6 * scale


def test_cube_level_pairs_match_oracle(cube):
    w, akl = cube
    lv = oracle_levels(w)
    for level, ids in [(1, [0, 3]), (2, [1])]:
        ctx = B.Context(B.make_config(w))
        y, y2, _, _, info = ctx.sample_level(level, 21, torch.tensor(ids))
        torch.cuda.synchronize()
        assert all(d["status"] == 0 for d in B.info_dicts(info))
        for r, i in enumerate(ids):
            yo, y2o = O.sample_pair_affine(lv[level], lv[level - 1], lv[0], akl, level, 21, i)
            assert np.abs(y[r].cpu().numpy() - yo).max() <= 1e-8
            assert np.abs(y2[r].cpu().numpy() - y2o).max() <= 1e-8
        ctx.close()
