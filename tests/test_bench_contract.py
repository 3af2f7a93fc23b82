"""The bench's JSON-line contract, on the CPU: the reference arm (the FP64 oracle timed on
the host) runs here on a short stream and must print one line with every required key."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "0", "--lines", "40"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "pixel-spectra scored/s" and d["unit"] == "pixel-spectra/s"
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] >= 3 and d["higher_is_better"] is True
    assert d["vs_baseline"] is None and d["config"]["workload"] == "precision_1024x448"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_roofline_work_and_peaks():
    """The factor's algorithmic work per line and the derived ceilings the bench divides by."""
    sys.path.insert(0, ROOT)
    import bench
    # B^3/3 + five 64-band diagonal blocks (64^3/3 x 4 + 14^3/3) at B = 270: 6.93 MFLOP
    assert abs(bench.factor_flops_per_line(270, 1) - (270 ** 3 + 4 * 64 ** 3 + 14 ** 3) / 3) < 1e-6
    assert abs(bench.factor_flops_per_line(270, 0) - 2 * 270 ** 3 / 3) < 1e-6
    assert abs(bench.fp64_peak_tflops(2070) - 1.25856) < 1e-9                    # 152 x 2070 MHz x 4
    assert abs(bench.ff_peak_tflops(2070) - 152 * 2070e6 * 128 * 2 / 12 / 1e12) < 1e-12


def test_kernel_rooflines_from_a_profile():
    """Per-kernel roofline entries: algorithmic work per step over the class's time per
    step, against the peak of the unit (and, for the tensor cores, the product scheme) that
    bounds each kernel; measured traffic per launch where a capture exists."""
    sys.path.insert(0, ROOT)
    import bench
    peaks = {"hbm_gbs": 6753.4, "bf16_tflops": 1849.2, "bf16_tflops_sustained": 1680.0, "source": "measured"}
    T, W, B = 8000, 1024, 448
    # two steps profiled: factor 4 launches of 2000 lines, syrk 4 launches, whitening 8
    prof = {"factor": (8, 8 * 30.0), "syrk": (8, 8 * 5.0), "whiten_score": (16, 16 * 2.0), "colsum": (8, 1.0)}
    r = bench.kernel_rooflines(prof, 2, T, W, B, 1, "fp32", 1, peaks, 2070.0)
    assert set(r) == {"factor", "syrk", "whiten_score", "colsum"}
    assert r["colsum"]["bound"] == "hbm" and abs(r["colsum"]["achieved"] - T * W * 2 * B / 0.0005 / 1e9) < 1e-6
    f = r["factor"]
    assert f["launches_per_step"] == 4 and abs(f["avg_launch_ms"] - 30.0) < 1e-12 and abs(f["ms_per_step"] - 120) < 1e-9
    assert abs(f["achieved"] - 8000 * bench.factor_flops_per_line(B, 1) / 0.120 / 1e12) < 1e-9
    assert f["bound"] == "alu" and abs(f["frac"] - f["achieved"] / bench.ff_peak_tflops(2070.0)) < 1e-12
    s = r["syrk"]
    assert s["bound"] == "tensor" and abs(s["achieved"] - T * W * B * (B + 1) / 0.020 / 1e12) < 1e-9
    # exact integer split: four BF16 products per product, against the sustained BF16 rate
    assert abs(s["peak"] - 1680.0 / 4) < 1e-12 and abs(s["frac"] - s["achieved"] / 420.0) < 1e-12
    assert abs(s["frac_of_bf16_peak"] - s["achieved"] / 1680.0) < 1e-12
    assert abs(s["traffic_algorithmic"] - T * W * 2 * B) < 1e-6 and s["traffic"] is None
    w = r["whiten_score"]
    assert w["bound"] == "alu" and abs(w["peak"] - bench.fp32_peak_tflops(2070.0)) < 1e-12
    assert abs(w["traffic_algorithmic"] - T * W * (2 * B + 5)) < 1e-6
    wb = bench.kernel_rooflines(prof, 2, T, W, B, 1, "bf16", 1, peaks, 2070.0)["whiten_score"]
    assert wb["bound"] == "tensor" and abs(wb["peak"] - 560.0) < 1e-9 and wb["operand_terms"] == 3
    # FP32 on the tensor cores (three-term operands): tensor bound, six products per product
    wx = bench.kernel_rooflines(prof, 2, T, W, B, 1, "fp32", 1, peaks, 2070.0, True)["whiten_score"]
    assert wx["bound"] == "tensor" and wx["operand_terms"] == 6 and abs(wx["peak"] - 280.0) < 1e-9
    assert abs(wx["issued_tflops"] - 6 * wx["achieved"]) < 1e-9
    assert bench.whitening_label(1, True) == "triangular solve, tensor cores"
    sp = bench.kernel_rooflines({"syrk_split": (4, 8.0)}, 2, T, W, B, 1, "fp32", 1, peaks, 2070.0)["syrk_split"]
    assert sp["bound"] == "hbm" and abs(sp["achieved"] - T * W * (2 * B + 4 * 128 * -(-B // 128)) / 0.004 / 1e9) < 1e-6
    # measured traffic: bytes per unit x units per step / launches per step, this workload only
    wt = bench.kernel_rooflines(prof, 2, T, W, B, 1, "fp32", 1, peaks, 2070.0, True,
                                "precision_1024x448")["whiten_score"]
    per_px = bench.DRAM_BYTES_PER_UNIT[("precision_1024x448", "fp32")]["whiten_score"][1]
    assert abs(wt["traffic"] - per_px * T * W / 8) < 1e-3
    # the tensor-core factor's three classes: their algorithmic parts add up to the Cholesky
    diag, trsm, upd = bench.factor_parts_per_line(B)
    blocks = [min(64, B - p) for p in range(0, B, 64)]
    assert abs((upd + diag + trsm - sum(b ** 3 / 3 for b in blocks)) - B ** 3 / 3) < 1e-3
    prof2 = {"factor_form": (8, 8.0), "factor_diag": (56, 10.0), "factor_panel": (48, 30.0),
             "factor_update": (48, 30.0)}
    r2 = bench.kernel_rooflines(prof2, 2, T, W, B, 1, "fp32", 1, peaks, 2070.0, True, "precision_1024x448")
    assert r2["factor_update"]["bound"] == "tensor" and r2["factor_panel"]["bound"] == "tensor"
    assert r2["factor_diag"]["bound"] == "alu" and abs(r2["factor_update"]["peak"] - 80.0) < 1e-9
    assert abs(r2["factor_diag"]["achieved"] - 8000 * diag / 0.005 / 1e12) < 1e-9
    assert abs(r2["factor_panel"]["achieved"] - 8000 * trsm / 0.015 / 1e12) < 1e-9
    assert abs(r2["factor_update"]["achieved"] - 8000 * upd / 0.015 / 1e12) < 1e-9
    per_line = bench.DRAM_BYTES_PER_UNIT[("precision_1024x448", "fp32")]["factor_update"][1]
    assert abs(r2["factor_update"]["traffic"] - per_line * 8000 / 24) < 1e-3
    assert abs(r2["factor_form"]["achieved"] - 8000 * B * (B + 1) / 2 * 16 / 0.004 / 1e9) < 1e-6
