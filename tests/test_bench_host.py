"""Host-side pieces of bench.py (no GPU): the HBM roofline arithmetic of the
3D global-memory sweep, the measured-peak lookup and the workload naming."""
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


def test_roofline_3d_bytes_and_fractions(bench, monkeypatch):
    monkeypatch.setattr(bench, "measured_hbm_peak", lambda: (5000.0, "test"))
    # 1e9 FP32 CG node-iterations, 2e8 FP64 ones, 1e8 Newton node-iterations
    r = bench.roofline_3d(cg64_ni=2e8, cg_ni=1.2e9, nw_ni=1e8, solve_ms=1000.0, dev_ms=500.0,
                          launches_per_step=7)
    nbytes = 164 * 1e9 + 328 * 2e8 + 560 * 1e8
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 5000.0
    assert r["achieved"] == pytest.approx(nbytes / 1.0 / 1e9)
    assert r["aggregate_gbs"] == pytest.approx(nbytes / 0.5 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 5000.0)
    assert bench.BYTES_CG32_NODE_3D == 27 * 4 + 14 * 4
    assert bench.BYTES_NEWTON_NODE_3D == 2 * (27 * 8 + 8 * 8)


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
