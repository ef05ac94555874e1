"""The group layout of the per-sample sweep (3D grids): G CTAs per sample that
form groups in arrival order and synchronise through bounded global-memory
barriers, so that a few samples of a large grid use every SM.

* forced on the 3D level-1 grid (64x64x16, several roots per step; G = 140 for
  one sample) against the oracle on the full grid for its first 4 steps, FP64
  and mixed;
* forced on the 3D level-0 grid with several samples per launch (groups of
  18 CTAs taking interleaved tickets) against the oracle;
* chosen automatically for one sample of the full-size 3D level 2 (G = 134)
  against the oracle-pinned global-memory cluster layout;
* inside a graph-launched two-level estimate (group launches ordered after one
  another inside the capture) against the cluster layouts;
* its bounded wait: a barrier that waits for one CTA too many runs out and
  every sample reports MLMC_ERR_TIMEOUT; the context stays usable."""
import numpy as np
import pytest

import oracle as O
from helpers import oracle_level
from paper_1911_06066_gb300 import binding as B
from paper_1911_06066_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GROUP = B.MLMC_LAYOUT_GROUP


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1911_06066_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def short_slab(steps_l1, levels=2):
    """The 3D slab workload cut to its first steps (T and m0 scaled alike)."""
    base = W.SLAB3D_4LVL
    m1 = base["m0"] * 2
    return dict(base, T=base["T"] * steps_l1 / m1, m0=steps_l1 // 2, levels=levels)


def test_group_layout_level1_full_grid_matches_oracle():
    w = short_slab(4)
    lv = oracle_level(w, 1)
    Zo = O.kl_field(3, w["L"], [64, 64, 16], w["sigma2"], w["ell"], w["M"], O.xi(0, 1, 3, w["M"]))[0]
    so, to, _ = O.solve_sample(lv, Zo)
    for precision in (B.MLMC_PREC_FP64, B.MLMC_PREC_MIXED):
        ctx = B.Context(B.make_config(w, precision))
        ctx.set_layout(1, GROUP)
        Z = ctx.kl_field(1, ctx.xi(0, 1, torch.tensor([3])))
        t, slab, info = ctx.solve(1, Z, slab=True)
        torch.cuda.synchronize()
        assert B.info_dicts(info)[0]["status"] == 0
        assert np.abs(slab[0].cpu().numpy() - so).max() <= 1e-8
        assert np.abs(t[0].cpu().numpy() - to).max() <= 1e-6 * W.SLAB3D_4LVL["T"]
        ctx.close()


def test_group_layout_several_samples_match_oracle():
    w = short_slab(8)
    ids = [0, 3, 5]
    ctx = B.Context(B.make_config(w, B.MLMC_PREC_FP64))
    ctx.set_layout(0, GROUP)
    Z = ctx.kl_field(0, ctx.xi(2, 0, torch.tensor(ids)))
    t, slab, info = ctx.solve(0, Z, slab=True)
    torch.cuda.synchronize()
    lv = oracle_level(w, 0)
    for r, i in enumerate(ids):
        assert B.info_dicts(info)[r]["status"] == 0
        Zo = O.kl_field(3, w["L"], [32, 32, 8], w["sigma2"], w["ell"], w["M"], O.xi(2, 0, i, w["M"]))[0]
        so, to, _ = O.solve_sample(lv, Zo)
        assert np.abs(slab[r].cpu().numpy() - so).max() <= 1e-8
        assert np.abs(t[r].cpu().numpy() - to).max() <= 1e-6 * w["T"]
    ctx.close()


def test_group_layout_full_size_level2_matches_cluster_layout():
    w = W.SLAB3D_4LVL
    out = {}
    for layout in (0, 116):   # automatic (the group layout for one sample), 16-CTA clusters
        ctx = B.Context(B.make_config(w, B.MLMC_PREC_FP64))
        ctx.set_layout(2, layout)
        Z = ctx.kl_field(2, ctx.xi(0, 2, torch.tensor([1])))
        t, _, info = ctx.solve(2, Z)
        torch.cuda.synchronize()
        assert B.info_dicts(info)[0]["status"] == 0
        out[layout] = t[0].cpu().numpy()
        ctx.close()
    assert np.abs(out[0] - out[116]).max() <= 1e-6 * w["T"]


def test_group_layout_inside_a_graph_launched_estimate():
    w = short_slab(8)
    st = torch.cuda.Stream()
    means = {}
    for layout in (GROUP, 116):
        ctx = B.Context(B.make_config(w, B.MLMC_PREC_FP64, use_graph=True))
        for l in range(2):
            ctx.set_layout(l, layout)
        with torch.cuda.stream(st):
            r = ctx.run([6, 3], seed=4, batch=3, stream=st)
        means[layout] = r["mean"]
        assert r["stats"]["failed"] == 0
        ctx.close()
    assert np.abs(means[GROUP] - means[116]).max() <= 1e-8 * w["T"]


def test_group_barrier_wait_runs_out_and_is_reported():
    w = short_slab(4)
    ctx = B.Context(B.make_config(w, B.MLMC_PREC_FP64))
    ctx.set_layout(0, GROUP)
    Z = ctx.kl_field(0, ctx.xi(1, 0, torch.tensor([0, 1])))
    ctx.check_timeout_path(2000)
    t, _, info = ctx.solve(0, Z)
    torch.cuda.synchronize()
    assert [d["status"] for d in B.info_dicts(info)] == [-4, -4]
    ctx.check_timeout_path(-1)
    t2, _, info2 = ctx.solve(0, Z)
    torch.cuda.synchronize()
    assert [d["status"] for d in B.info_dicts(info2)] == [0, 0]
    ref = B.Context(B.make_config(w, B.MLMC_PREC_FP64))
    t3, _, _ = ref.solve(0, Z)
    torch.cuda.synchronize()
    assert np.abs(t2.cpu().numpy() - t3.cpu().numpy()).max() <= 1e-6 * w["T"]
    ctx.close()
    ref.close()


def test_level1_full_run_every_step_a_root_in_both_layouts():
    """On the 64x64x16 grid (c dt max r' = 2.37) some steps pass so close to a
    saddle of the step energy that the rounding order of the reductions picks
    the basin: the cluster and the group layout can end such a step in roots
    that put the front one or two steps apart at a few nodes.  What is unique
    is checked over the full 64-step run: in both layouts every step satisfies
    its residual (Eq. mono_disc) to the Newton tolerance."""
    w = W.SLAB3D_4LVL
    for layout in (116, GROUP):
        ctx = B.Context(B.make_config(w, B.MLMC_PREC_FP64, newton_max=40000))
        ctx.set_layout(1, layout)
        Z = ctx.kl_field(1, ctx.xi(5, 1, torch.tensor([0])))
        t, slab, info = ctx.solve(1, Z, slab=True)
        torch.cuda.synchronize()
        assert B.info_dicts(info)[0]["status"] == 0, B.info_dicts(info)
        _, rmax = ctx.slab_residual(1, Z, slab, full=False)
        assert rmax.item() <= 1e-8, rmax.item()
        ctx.close()


def test_capped_group_launches_inside_an_estimate():
    """20 samples of the 64x64x16 level in one estimate: the group layout
    caps a launch at the samples whose groups of >= 32 CTAs are resident at
    once (9 on GB300), so the level runs as several group launches one after
    another; the mean equals that of one 16-CTA cluster launch."""
    w = short_slab(4)
    st = torch.cuda.Stream()
    means = {}
    for layout in (0, 116):
        ctx = B.Context(B.make_config(w, B.MLMC_PREC_FP64, use_graph=True))
        for l in range(2):
            ctx.set_layout(l, layout)
        with torch.cuda.stream(st):
            r = ctx.run([4, 20], seed=6, batch=64, stream=st)
        assert r["stats"]["failed"] == 0
        means[layout] = r["mean"]
        ctx.close()
    assert np.abs(means[0] - means[116]).max() <= 1e-6 * w["T"]
