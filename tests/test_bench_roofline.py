"""The benchmark's roofline arithmetic on made-up stage times and counts, recomputed here
from the definitions: achieved work per second against the peak for the dominant stage
and for each HBM-bound stage, the derived FP32 peak when no probe ran, and the
whole-path roofline; and the per-pair flop constants against the totals of the frozen
operation table (docs/flops.md)."""
import os
import re
from types import SimpleNamespace

import pytest

import bench

STAGES = {"binning": 0.2, "emit": 0.25, "sort": 0.3, "composite_fwd": 1.5, "composite_bwd": 1.6, "finalize": 0.03}
N_G = 2_457_600
STATS = {"n_keys": 40_000_000, "n_pairs": 140_000_000}
SCENE = SimpleNamespace(n_gaussians=N_G, n_pixels=N_G)
PEAKS = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}
FP32 = {"measured_tflops": 78.0}


def test_dominant_stage_is_the_backward_against_the_measured_fp32_peak():
    r = bench.roofline(STAGES, STATS, SCENE, PEAKS, "measured", bwd_kernel="k_composite_bwdl", fp32=FP32)
    assert (r["kernel"], r["bound"], r["unit"]) == ("k_composite_bwdl", "alu", "TFLOP/s")
    achieved = 140e6 * 77 / 1.6e-3 / 1e12              # pairs x flops per pair / seconds
    assert r["achieved"] == pytest.approx(achieved, abs=1e-3)
    assert r["peak"] == pytest.approx(78.0)
    assert r["frac"] == pytest.approx(achieved / 78.0, abs=1e-4)
    assert r["avg_ms"] == pytest.approx(1.6)


def test_forward_without_a_probe_takes_the_derived_fp32_peak():
    r = bench.roofline(STAGES, STATS, SCENE, PEAKS, "measured", name="composite_fwd")
    peak = 152 * 128 * 2 * 2070e6 / 1e12                # SMs x FP32 lanes x 2 flop x clock
    achieved = 140e6 * 29 / 1.5e-3 / 1e12
    assert r["kernel"] == "k_composite_fwd"
    assert r["peak"] == pytest.approx(peak, abs=0.01)
    assert r["frac"] == pytest.approx(achieved / peak, abs=1e-4)


@pytest.mark.parametrize("name,byts,kernel", [
    ("sort", 40e6 * 16, "k_sort_tiles_bucket"),                  # 8 B read + 8 B written per key
    ("emit", N_G * 40 + 40e6 * 8, "k_emit"),
    ("binning", N_G * 60, "k_project_count"),
    ("finalize", N_G * 68, "k_finalize"),
])
def test_hbm_bound_stages(name, byts, kernel):
    r = bench.roofline(STAGES, STATS, SCENE, PEAKS, "measured", fp32=FP32, name=name)
    gbs = byts / (STAGES[name] * 1e-3) / 1e9
    assert (r["kernel"], r["bound"], r["unit"]) == (kernel, "hbm", "GB/s")
    assert r["achieved"] == pytest.approx(gbs, abs=1e-3)
    assert r["frac"] == pytest.approx(gbs / 6800.0, abs=1e-4)


def test_whole_path_roofline():
    p = bench.path_roofline(STAGES, STATS, SCENE, PEAKS, FP32)
    b = 80 * N_G + 24 * 40e6 + 56 * N_G                           # per Gaussian, per key, per view pixel
    f = (29 + 77) * 140e6
    t_hbm, t_fp32 = b / 6800e9 * 1e3, f / 78e12 * 1e3
    t = sum(STAGES.values())
    assert (p["bytes_alg"], p["flops_alg"]) == (int(b), int(f))
    assert p["t_roof_ms"] == pytest.approx(max(t_hbm, t_fp32), abs=1e-4)
    assert p["t_measured_ms"] == pytest.approx(t, abs=1e-4)
    assert p["frac"] == pytest.approx(max(t_hbm, t_fp32) / t, abs=1e-4)
    assert p["bound"] == ("hbm" if t_hbm >= t_fp32 else "alu")


def test_flop_constants_match_the_operation_table():
    text = open(os.path.join(os.path.dirname(__file__), "..", "docs", "flops.md")).read()
    fwd = re.search(r"## Forward, per contributing pair: .*= (\d+)", text)
    bwd = re.search(r"## Backward, per contributing pair: .*= (\d+)", text)
    assert fwd and bwd
    assert (int(fwd.group(1)), int(bwd.group(1))) == (bench.FLOPS_FWD_PAIR, bench.FLOPS_BWD_PAIR)
