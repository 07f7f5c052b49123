"""Host logic of bench.py that needs no GPU: the k_push source hash that gates
the recorded DRAM traffic covers the kernel source only, and the roofline
arithmetic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_source_text_drops_host_only_sections():
    text = ("// preamble\nconstexpr int A = 1;\n"
            "// --------------------------------------------------------------------------- handle\n"
            "struct pic_t { int host_only; };\n"
            "// --------------------------------------------------------------------------- device helpers\n"
            "__device__ inline int f() { return 1; }\n"
            "// --------------------------------------------------------------------------- host entry points\n"
            "int host_function(pic_t *h);\n")
    kept = bench.kernel_source_text(text)
    assert "constexpr int A = 1;" in kept and "__device__ inline int f()" in kept
    assert "host_only" not in kept and "host_function" not in kept


def test_source_hash_is_stable_and_covers_the_header_sections():
    h = bench.push_source_sha()
    assert len(h) == 16 and h == bench.push_source_sha()
    with open(os.path.join(ROOT, "paper_1308_2590_gb300/csrc/pic_internal.cuh")) as f:
        text = f.read()
    kept = bench.kernel_source_text(text)
    assert "__device__ inline void particle_moments_c" in kept      # device helpers are hashed
    assert "struct pic_t {" not in kept                              # the handle is not
    assert "int push_work_list(pic_t *h);" not in kept               # nor the host entry points


def _r(push_ms_per_step, steps, n):
    return {"kernel_ms": [push_ms_per_step * steps, 0.0, 0.0, 0.0], "n_local": n}


def test_roofline_fp32_is_algorithmic_bytes_over_launch_time():
    n, steps, t = 6553600, 200, 0.26
    peaks = {"hbm_gbs": 6762.3}
    ro = bench.roofline(_r(t, steps, n), "fp32", "atomic", steps, peaks, "measured")
    gbs = 52 * n / (t * 1e-3) / 1e9        # 28 B read + 24 B written per particle-step
    assert ro["bound"] == "hbm" and ro["unit"] == "GB/s" and ro["peak"] == 6762.3
    assert abs(ro["achieved"] - gbs) < 1e-9 * gbs and abs(ro["frac"] - gbs / 6762.3) < 1e-12
    assert "measured" in ro["peak_source"]
    # traffic: the captured DRAM bytes per particle x the particles of one launch, for this source only
    if bench.PUSH_SOURCE_SHA == bench.push_source_sha():
        assert ro["traffic"] == bench.PUSH_TRAFFIC_PER_PARTICLE["fp32"] * n
    assert bench.roofline(_r(t, steps, n), "fp32", "deterministic", steps, peaks, "measured")["traffic"] is None


def test_roofline_fp64_is_flops_over_the_fp64_peak():
    n, steps, t = 6553600, 200, 3.16
    ro = bench.roofline(_r(t, steps, n), "fp64", "atomic", steps, {"hbm_gbs": 6762.3}, "measured")
    tf = 250 * n / (t * 1e-3) / 1e12
    assert ro["bound"] == "alu" and ro["unit"] == "TFLOP/s"
    assert abs(ro["peak"] - 2 * 2 * 152 * 2.070e9 / 1e12) < 1e-12    # 2 DFMA/clk/SM, 152 SMs, 2070 MHz
    assert abs(ro["achieved"] - tf) < 1e-9 * tf and abs(ro["frac"] - tf / ro["peak"]) < 1e-12
    assert abs(ro["hbm_frac"] - 96 * n / (t * 1e-3) / 1e9 / 6762.3) < 1e-12


def test_traffic_is_null_for_another_kernel_source(monkeypatch):
    monkeypatch.setattr(bench, "PUSH_SOURCE_SHA", "0" * 16)
    for prec in ("fp32", "fp64"):
        assert bench.roofline(_r(1.0, 10, 1000), prec, "atomic", 10, {"hbm_gbs": 6762.3}, "measured")["traffic"] is None


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    root = bench.ROOT
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))   # a tree without the generated file
    peaks, src = bench.measured_peaks()
    monkeypatch.setattr(bench, "ROOT", root)            # the kernel sources for the traffic gate
    assert src == "fallback" and peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops"] == 1900.0
    ro = bench.roofline(_r(0.26, 200, 6553600), "fp32", "atomic", 200, peaks, src)
    assert ro["peak"] == 6800.0 and "fallback" in ro["peak_source"] and "no MEASURED_PEAKS.json" in ro["peak_source"]
