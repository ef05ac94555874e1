"""Host-side pieces of bench.py (no GPU): the per-level ALU bounds and the HBM
roofline arithmetic of the global-memory sweep, the measured-peak lookup and
the workload naming."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _per_level():
    # two grid levels' counters of one step: CG / nonlinear / FP64-CG node-iterations
    return [dict(solve_ms=400.0, solve_launches=2, cg_node_iters=1.2e9, newton_node_iters=1e8,
                 cg64_node_iters=2e8, truncations=0, halvings=5, not_converged=0),
            dict(solve_ms=100.0, solve_launches=1, cg_node_iters=1e8, newton_node_iters=1e7,
                 cg64_node_iters=1e8, truncations=0, halvings=0, not_converged=0)]


def test_level_bounds_alu_time(bench):
    peaks = {"fp64_tflops": 1.0, "fp32_tflops": 50.0}
    lv = bench.level_bounds(_per_level(), 2, peaks)
    f64 = (32 * 1e8 + 31 * 2e8) / 2
    f32 = 31 * 1e9 / 2
    assert lv[0]["solve_ms"] == 200.0
    assert lv[0]["fp64_gflop"] == pytest.approx(f64 * 1e-9)
    assert lv[0]["fp32_gflop"] == pytest.approx(f32 * 1e-9)
    t = f64 / 1e12 + f32 / 50e12
    assert lv[0]["alu_bound_ms"] == pytest.approx(t * 1e3)
    assert lv[0]["frac"] == pytest.approx(t * 1e3 / 200.0)
    r = bench.roofline_2d(lv, 300.0, peaks, True)
    # the dominant level is level 0; FP64-equivalent flops over its time
    eq = (f64 + f32 * 1.0 / 50.0)
    assert r["bound"] == "alu" and r["peak"] == 1.0
    assert r["achieved"] == pytest.approx(eq / 0.2 / 1e12)
    assert r["frac"] == pytest.approx(lv[0]["frac"])


def test_roofline_3d_bytes_and_fractions(bench, monkeypatch):
    monkeypatch.setattr(bench, "measured_hbm_peak", lambda: (5000.0, "test"))
    peaks = {"fp64_tflops": 1.0, "fp32_tflops": 50.0}
    per = _per_level()
    lv = bench.add_hbm_bytes(bench.level_bounds(per, 1, peaks), per, 1)
    nbytes = 112 * 1e9 + 224 * 2e8 + 352 * 1e8
    assert lv[0]["hbm_gb"] == pytest.approx(nbytes * 1e-9)
    r = bench.roofline_3d(lv, 1000.0, peaks)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 5000.0
    assert r["achieved"] == pytest.approx(nbytes / 0.4 / 1e9)
    tot = nbytes + 224 * 1e8 + 352 * 1e7
    assert r["aggregate_gbs"] == pytest.approx(tot / 1.0 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 5000.0)
    # every level carries its own fraction; the finest level's is reported too
    assert [v["hbm_frac"] for v in lv] == pytest.approx([v["hbm_gbs"] / 5000.0 for v in lv])
    assert r["finest_level_frac"] == pytest.approx(lv[-1]["hbm_gbs"] / 5000.0)
    # each symmetric coupling pair stored once: 14 couplings per node
    assert bench.BYTES_CG32_NODE_3D == 14 * 4 + 14 * 4
    assert bench.BYTES_NEWTON_NODE_3D == 2 * (14 * 8 + 8 * 8)


def test_measured_peak_lookup(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, src = bench.measured_hbm_peak()
    assert peak == 6800.0 and src.startswith("fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6794.5}))
    peak, src = bench.measured_hbm_peak()
    assert peak == 6794.5 and src.startswith("measured")


def test_workload_grid_names(bench):
    from paper_1911_06066_gb300 import workloads as W
    assert bench.grids_of(W.MLMC2D_3LVL) == "32x32/64x64/128x128"
    assert bench.grids_of(W.SLAB3D_4LVL) == "32x32x8/64x64x16/128x128x32/256x256x64"


def test_cpu_estimate_extrapolation(bench):
    w = {"N": [10, 4, 2]}
    assert bench.cpu_estimate_seconds(w, [1.0, 2.0, 5.0], cores=2) == pytest.approx((10 + 8 + 10) / 2)
