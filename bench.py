#!/usr/bin/env python
"""Throughput / latency benchmark of streaming RX on one GB300 (or N replicas).

Workload (default): the precision form, 1024 pixels x 448 bands x 8000 lines of uint16
12-bit DN pushed in batches of 2000, EXCLUSIVE running statistics (each line scored
against all earlier lines, Sec. 6.1's line-based form of the global RX of Sec. 3.3), ABS
threshold. One step = restart the stream and push all 8000 lines (resident in HBM)
through the C ABI, then read every score and mask back into device memory.

Printed: one JSON line whose headline is the FP32 path (the paper's detector computes in
FP32), in pixel-spectra scored / s (whole job); the same metric end to end from pinned
host memory; the BF16 path and the FP32 path with the FP64 factor on the same workload and
step count beside it, each with its error against the FP64 oracle on a sampled line;
p50/p99 single-line latency; roofline entries of the factor, covariance and whitening
kernels timed live with CUDA events on the launching stream; clocks sampled during the
timed region; and the FP64 oracle timed on a bounded sample on the host.

``--impl reference`` times the oracle itself (the only reference that exists).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # the whole stream is one batch: one launch per kernel, one wave tail per step
    "stream_640x270": dict(width=640, bands=270, lines=4000, batch=4000),
    "precision_1024x448": dict(width=1024, bands=448, lines=8000, batch=2000),
    # the paper's own line (Sec. 3.2): 900 samples x 300 raw bands, bands 10.. kept and binned by
    # four into 70 on the device (the front end)
    "frontend_900x300": dict(width=900, bands=70, lines=4000, batch=4000, raw_bands=300, band_first=10,
                             band_bin=4),
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d.get("hbm_gbs", 6800.0), bf16_tflops=d.get("bf16_tflops", 1900.0),
                    bf16_tflops_sustained=d.get("bf16_tflops_sustained", 1700.0), source="measured",
                    sm_max_mhz=d.get("sm_max_mhz", 2070.0))
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, source="fallback",
                sm_max_mhz=2070.0)


# DRAM bytes per unit (line or pixel) of a kernel class from one ncu capture of the same
# kernels on a 256-line batch of the precision_1024x448 workload in the FP32 form
# (dram__bytes_read.sum + dram__bytes_write.sum summed over the class's launches of one
# batch, divided by its lines or pixels); per-launch traffic = that x units per step /
# launches per step. Work and traffic per unit do not depend on the batch size. Only this
# workload and form, and only kernels unchanged since the capture, have an entry; the rest
# report null.
DRAM_BYTES_PER_UNIT = {
    ("precision_1024x448", "fp32"): {
        "factor_update": ("line", 3.552e6),
        "factor_panel": ("line", 1.947e6),
        "factor_diag": ("line", 0.1495e6),
        "prefix_cov": ("line", 2.172e6),
        "syrk": ("px", 2769.0),
        "syrk_split": ("px", 2748.0),
        "whiten_score": ("px", 1655.0),
    },
}

# BF16 tensor-core products issued per algorithmic product by each contraction's exact or
# extended-precision scheme: the peak of that arithmetic on this GPU is the BF16 peak divided
# by it (the kernel's own dtype; reported beside the plain BF16 fraction).
TERMS = {
    "factor_update": 21,    # six base-256 digits per operand, levels t + u <= 5
    "factor_panel": 21,
    "syrk": 4,              # x' = 64 h + r: HH, HR, RH, RR
    "whiten_fp32": 6,       # three BF16 terms per operand, products with t + u <= 2
    "whiten_bf16": 3,       # a_hi h_hi + a_hi h_lo + a_lo h_hi
    "whiten_fp16": 2,
}


def factor_flops_per_line(B, form):
    """Algorithmic flops of one line's factorisation: the Cholesky factor (B^3 / 3)
    plus the full triangular inverse (B^3 / 3) for the explicit-inverse form, or plus only
    the inverses of the 64 x 64 diagonal blocks (b^3 / 3 each) for the triangular solve."""
    if form == 0:
        return 2.0 * B ** 3 / 3.0
    blocks = [min(64, B - b) for b in range(0, B, 64)]
    return B ** 3 / 3.0 + sum(b ** 3 / 3.0 for b in blocks)


# FP64 and FP32 SIMT peaks derived from unit counts x clock (no measured figure exists):
# 152 SMs x 2070 MHz x (4 FP64 flops / clk / SM, i.e. the 1.25 TF/s nominal) and
# x (128 FP32 lanes x 2 flops / clk / SM).
def fp64_peak_tflops(mhz):
    return 152 * mhz * 1e6 * 4 / 1e12


def fp32_peak_tflops(mhz):
    return 152 * mhz * 1e6 * 256 / 1e12


# The factor's O(B^3) updates run in float-float: one multiply-subtract of two pairs into a
# compensated sum is 12 FP32-pipe instructions (product, three FMAs for its error, six for
# the two-sum, two to gather the errors) for 2 flops of the algorithm, so its ALU ceiling is
# the FP32 instruction rate x 2 / 12.
FF_INSTR_PER_MAC = 12


def ff_peak_tflops(mhz):
    return 152 * mhz * 1e6 * 128 * 2 / FF_INSTR_PER_MAC / 1e12


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def oracle_sample(lines, t_list, gain, offset):
    """Time the FP64 oracle scoring the given lines of the stream (EXCLUSIVE)."""
    import oracle
    from oracle import rx as orx
    t0 = time.perf_counter()
    px = 0
    for t in t_list:
        d, st = orx.stream_rx_line(lines, t, oracle.EXCLUSIVE, gain=gain, offset=offset)
        px += d.size
    return px, time.perf_counter() - t0


def oracle_sample_scores(lines, t, gain, offset):
    """The FP64 oracle scoring line t of the stream (EXCLUSIVE): pixels, seconds, scores."""
    import oracle
    from oracle import rx as orx
    t0 = time.perf_counter()
    d, st = orx.stream_rx_line(lines, t, oracle.EXCLUSIVE, gain=gain, offset=offset)
    return d.size, time.perf_counter() - t0, d


# Score tolerances and mask margins of the parity tests (relative error |d - ref| / max(ref, 1)).
TOL = {"fp32": 1e-4, "bf16": 1e-2, "fp16": 1e-2}
MARGIN = {"fp32": 2e-4, "bf16": 2e-2, "fp16": 2e-2}


def accuracy_vs_oracle(s, m, ref, B, prec, t):
    """Error of one arm's scores of line t against the oracle's, and mask disagreement."""
    import numpy as np
    s = np.asarray(s, np.float64)
    ok = np.isfinite(ref)
    e = np.abs(s[ok] - ref[ok]) / np.maximum(ref[ok], 1.0)
    tau = B + 6 * math.sqrt(2 * B)
    band = np.abs(ref - tau) <= MARGIN[prec] * tau
    diff = (np.asarray(m).astype(bool) != (ref > tau))
    return {"line": int(t), "pixels": int(ok.sum()), "max_rel_err": float(e.max()) if e.size else None,
            "p999_rel_err": float(np.percentile(e, 99.9)) if e.size else None, "tolerance": TOL[prec],
            "mask_diff_outside_margin": int((diff & ~band).sum()), "mask_diff_total": int(diff.sum())}


def factor_parts_per_line(B):
    """Algorithmic flops of one line's blocked factorisation in 64-column panels (the
    tensor-core factor): per panel k (kb columns, r rows below) the diagonal block's Cholesky
    kb^3/3 and inverse kb^3/3 (the diagonal-block kernel), the rows' triangular solve r kb^2
    (the panel kernel), and the rest of the Cholesky's B^3/3, the trailing updates (the update
    kernel)."""
    diag, trsm, chol_panel = 0.0, 0.0, 0.0
    for p0 in range(0, B, 64):
        kb = min(64, B - p0)
        r = B - p0 - kb
        diag += 2 * kb ** 3 / 3.0
        trsm += r * kb * kb
        chol_panel += kb ** 3 / 3.0 + r * kb * kb
    return diag, trsm, B ** 3 / 3.0 - chol_panel


def whitening_label(form, tc):
    """How the arm whitens: the form (Sec. 3.3) and the units its contraction runs on."""
    return ("triangular solve" if form else "explicit inverse") + (", tensor cores" if tc else ", SIMT cores")


def tensor_peak(peaks, terms):
    """Peak of a contraction whose scheme issues `terms` BF16 products per algorithmic product,
    timed inside full steps: the measured sustained BF16 rate divided by `terms`."""
    return peaks["bf16_tflops_sustained"] / terms


def kernel_rooflines(prof, prof_steps, T, W, B, form, prec, every, peaks, mhz, tc_whiten=None, workload=None):
    """Roofline entries of the factor (whole, or its covariance, diagonal-block, panel and
    update kernels), covariance (SYRK and its split) and whitening kernels of one arm:
    algorithmic work per step (per-unit figures x units per step) over the kernel class's
    CUDA-event time per step (measured inside full steps), against the peak of the unit and
    dtype that bound it. A tensor-core contraction computing exact or extended-precision
    products from BF16 terms takes the sustained BF16 peak divided by the BF16 products it
    issues per algorithmic product; `frac_of_bf16_peak` gives the plain BF16 fraction."""
    out = {}
    px_step = T * W
    lines = T / max(1, every)                    # factorisations per step
    ffp = ff_peak_tflops(mhz)
    sus = peaks["bf16_tflops_sustained"]
    src_t = f"{peaks['source']} bf16 sustained"
    dram = DRAM_BYTES_PER_UNIT.get((workload, prec), {})
    for name, (n, tot) in prof.items():
        if n == 0 or name not in ("factor", "factor_form", "factor_diag", "factor_panel", "factor_update", "syrk",
                                   "syrk_split", "whiten_score", "prefix_cov", "colsum"):
            continue
        ms = tot / prof_steps
        r = None
        if name == "factor":
            work = lines * factor_flops_per_line(B, form)
            ach = work / (ms / 1e3) / 1e12
            r = {"bound": "alu", "achieved": ach, "peak": ffp, "unit": "TFLOP/s", "frac": ach / ffp,
                 "traffic_algorithmic": lines * (B * B * 8 + B * 8 + pad64(B) ** 2 * 4),
                 "kernel": "factor (CUDA cores: Cholesky + inverses of the 64 x 64 diagonal blocks)" if form
                           else "factor (Cholesky + triangular inverse)",
                 "work_per_step": (f"{lines:.0f} lines x (B^3/3 + sum of 64-block b^3/3) flop" if form
                                   else f"{lines:.0f} lines x 2B^3/3 flop"),
                 "peak_source": "derived: 152 SMs x %.0f MHz x 128 FP32 lanes x 2 flop / 12 FP32 instructions "
                                "per float-float multiply-subtract" % mhz,
                 "fp64_peak_derived": fp64_peak_tflops(mhz), "frac_of_fp64_peak": ach / fp64_peak_tflops(mhz)}
        elif name == "factor_diag":
            work = lines * factor_parts_per_line(B)[0]
            ach = work / (ms / 1e3) / 1e12
            r = {"bound": "alu", "achieved": ach, "peak": ffp, "unit": "TFLOP/s", "frac": ach / ffp,
                 "kernel": "factor diagonal blocks (64 x 64 Cholesky + inverse, float-float on the CUDA cores)",
                 "work_per_step": f"{lines:.0f} lines x sum over panels 2 kb^3/3 flop",
                 "peak_source": "derived: 152 SMs x %.0f MHz x 128 FP32 lanes x 2 flop / 12 FP32 instructions "
                                "per float-float multiply-subtract" % mhz}
        elif name in ("factor_panel", "factor_update"):
            upd = name == "factor_update"
            work = lines * factor_parts_per_line(B)[2 if upd else 1]
            ach = work / (ms / 1e3) / 1e12
            pk = tensor_peak(peaks, TERMS[name])
            r = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                 "kernel": ("factor trailing updates" if upd else "factor panels (rows below the diagonal blocks: "
                            "L_ik = A_ik L_kk^-T)") + " on tcgen05, six-digit exact BF16 splits: 21 digit-product "
                            "MMAs per float-float-accurate product",
                 "work_per_step": (f"{lines:.0f} lines x (B^3/3 - panel Cholesky flops) algorithmic flop" if upd
                                   else f"{lines:.0f} lines x sum over panels r kb^2 algorithmic flop"),
                 "issued_tflops": TERMS[name] * ach, "frac_of_bf16_peak": ach / sus,
                 "peak_source": f"{src_t} / {TERMS[name]} (BF16 products per product)"}
        elif name == "syrk_split":
            byts = px_step * (2 * B + 4 * (-(-B // 128) * 128))
            ach = byts / (ms / 1e3) / 1e9
            r = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": ach / peaks["hbm_gbs"], "kernel": "SYRK operand split (uint16 DN in, BF16 h and r "
                 "blocks out in the tensor-core operand layout)",
                 "work_per_step": f"{px_step} px x (2 B + 4 x B rounded up to 128) bytes",
                 "peak_source": peaks["source"]}
        elif name == "prefix_cov":
            byts = T * B * (B + 1) / 2 * 16
            ach = byts / (ms / 1e3) / 1e9
            r = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": ach / peaks["hbm_gbs"], "kernel": "running covariance sums per line (FP64 in; FP64, or "
                 "for the tensor-core factor the formed float-float covariance, out)",
                 "work_per_step": f"{T} lines x B(B+1)/2 x 16 bytes", "peak_source": peaks["source"]}
        elif name == "colsum":
            byts = px_step * 2 * B
            ach = byts / (ms / 1e3) / 1e9
            r = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": ach / peaks["hbm_gbs"], "kernel": "per-line band sums (uint16 DN in)",
                 "work_per_step": f"{px_step} px x 2 B bytes", "peak_source": peaks["source"]}
        elif name == "factor_form":
            byts = lines * B * (B + 1) / 2 * 16
            ach = byts / (ms / 1e3) / 1e9
            r = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": ach / peaks["hbm_gbs"], "kernel": "covariance formation (FP64 sums in, float-float out)",
                 "work_per_step": f"{lines:.0f} lines x B(B+1)/2 x 16 bytes", "peak_source": peaks["source"]}
        else:
            flops = px_step * B * (B + 1)               # B(B+1)/2 multiply-adds per pixel
            byts = px_step * (2 * B + (5 if name == "whiten_score" else 0))
            ach = flops / (ms / 1e3) / 1e12
            tcw = (prec != "fp32") if tc_whiten is None else tc_whiten
            if name == "whiten_score" and not tcw:
                pk, bound, src, terms = fp32_peak_tflops(mhz), "alu", \
                    "derived: 152 SMs x %.0f MHz x 128 FFMA x 2" % mhz, None
            else:
                terms = TERMS["syrk"] if name == "syrk" else TERMS["whiten_" + prec]
                pk, bound = tensor_peak(peaks, terms), "tensor"
                src = f"{src_t} / {terms} (BF16 products per product)"
            r = {"bound": bound, "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                 "traffic_algorithmic": byts, "kernel": name, "work_per_step": f"{px_step} px x B(B+1) flop",
                 "peak_source": src, "hbm_achieved_gbs": byts / (ms / 1e3) / 1e9,
                 "hbm_frac": byts / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}
            if terms:
                r["operand_terms"] = terms
                r["issued_tflops"] = terms * ach
                r["frac_of_bf16_peak"] = ach / sus
        unit = dram.get(name)
        if unit:
            per_step = unit[1] * (lines if unit[0] == "line" else px_step)
            r["traffic"] = per_step / (n / prof_steps)
            r["traffic_source"] = f"ncu DRAM bytes per {unit[0]} of a 256-line batch x {unit[0]}s per launch"
        else:
            r["traffic"] = None
        r["ms_per_step"] = ms
        r["launches_per_step"] = n / prof_steps
        r["avg_launch_ms"] = tot / n
        out[name] = r
    return out


def pad64(b):
    return (b + 63) // 64 * 64


def gpu_local_cpus(index):
    """CPUs next to GPU `index` (its sysfs local_cpulist) that this process may use."""
    try:
        import torch
        p = torch.cuda.get_device_properties(index)
        path = "/sys/bus/pci/devices/%04x:%02x:%02x.0/local_cpulist" % (p.pci_domain_id, p.pci_bus_id,
                                                                        p.pci_device_id)
        cpus = set()
        for part in open(path).read().strip().split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        return sorted(cpus & os.sched_getaffinity(0))
    except Exception:
        return []


def bind_near_gpu(index):
    """Run on the GPU's local CPUs, so that host buffers (first touched by this process)
    sit on the GPU's NUMA node and host<->device copies take the direct link."""
    cpus = gpu_local_cpus(index)
    if cpus and set(cpus) != os.sched_getaffinity(0):
        os.sched_setaffinity(0, cpus)
        how = "bound to the GPU's local CPUs"
    else:
        how = "all GPU-local" if cpus else "GPU locality unknown"
    return "%d CPUs (%s)" % (len(os.sched_getaffinity(0)), how)


def max_over_ranks(ms, dist, device):
    """Slowest rank's time (replicas run independent streams; this is the only collective)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(px_per_rank_step, world, ms):
    """Whole-job pixel-spectra per second: every rank scores its own stream."""
    return px_per_rank_step * world / (ms / 1e3)


def run_serving(hs, device, precision, seconds, warm_s, pool_lines=96, seed_offset=0):
    """16 concurrent streams with Poisson line arrivals through the serving engine.

    Streams follow gen.serving_streams (widths {320,640,1024}, bands {128,270,448}, rates
    U[100,300] lines/s). Each stream cycles through a pool of generated lines. Latency =
    scores on the host minus the line's scheduled arrival (open loop: submissions follow
    the schedule, not completions). Returns a dict for the JSON line.
    """
    import threading

    import numpy as np
    from gen import PushbroomScene, serving_streams

    specs = serving_streams(16)
    pools, scenes = [], []
    for i, sp in enumerate(specs):
        sc = PushbroomScene(sp["width"], sp["bands"], seed=sp["seed"] + seed_offset)
        scenes.append(sc)
        pools.append(sc.lines(0, pool_lines))
    rng = np.random.default_rng(20260213 + 4)
    total = warm_s + seconds
    sched = []  # (time, stream, line index)
    for i, sp in enumerate(specs):
        t, k = 0.0, 0
        while True:
            t += rng.exponential(1.0 / sp["rate"])
            if t >= total:
                break
            sched.append((t, i, k))
            k += 1
    sched.sort()
    n_lines = [sum(1 for e in sched if e[1] == i) for i in range(len(specs))]

    rc, eng = hs.hsad_engine_create(device, 0)
    assert rc == hs.HSAD_OK
    sids = []
    for i, sp in enumerate(specs):
        cfg = hs.make_config(sp["width"], sp["bands"], precision=precision, gain=scenes[i].gain,
                             offset=scenes[i].offset, max_batch_lines=32, result_lines=max(8192, n_lines[i] + 64),
                             device=device)
        rc, sid = hs.hsad_engine_open(eng, cfg)
        assert rc == hs.HSAD_OK, hs.hsad_status_string(rc)
        sids.append(sid)
    t_sched = [np.zeros(n) for n in n_lines]
    t_done = [np.zeros(n) for n in n_lines]
    for (t, i, k) in sched:
        t_sched[i][k] = t
    start = time.perf_counter() + 0.2

    def waiter(i):
        W = specs[i]["width"]
        s = np.empty((1, W), np.float32)
        m = np.empty((1, W), np.uint8)
        for k in range(n_lines[i]):
            while time.perf_counter() < start + t_sched[i][k]:  # not yet submitted
                time.sleep(0.0002)
            rc = hs.hsad_engine_results(eng, sids[i], k, 1, s, m, 60000)
            t_done[i][k] = time.perf_counter() - start

    switch = sys.getswitchinterval()
    sys.setswitchinterval(1e-4)                         # GIL hand-over well below a line period
    threads = [threading.Thread(target=waiter, args=(i,), daemon=True) for i in range(len(specs))]
    for th in threads:
        th.start()
    for (t, i, k) in sched:
        while True:                                     # sleep, do not spin: the waiters need the GIL
            dt = start + t - time.perf_counter()
            if dt <= 0:
                break
            time.sleep(min(dt, 0.0002))
        line = pools[i][k % pool_lines:k % pool_lines + 1]
        hs.hsad_engine_submit(eng, sids[i], line, 1)
    for th in threads:
        th.join()
    sys.setswitchinterval(switch)
    err, lines_pushed, pushes, max_batch = hs.hsad_engine_counters(eng)
    hs.hsad_engine_destroy(eng)

    lat_all, px, over = [], 0, []
    by_b, ok_streams = {}, 0
    for i, sp in enumerate(specs):
        sel = t_sched[i] >= warm_s
        lat = (t_done[i][sel] - t_sched[i][sel]) * 1e3
        lat_all.append(lat)
        px += int(sel.sum()) * sp["width"]
        by_b.setdefault(sp["bands"], []).append(lat)
        if lat.size and np.percentile(lat, 99) < 1e3 / sp["rate"]:
            ok_streams += 1
        elif lat.size:
            over.append({"stream": i, "width": sp["width"], "bands": sp["bands"],
                         "p99_ms": round(float(np.percentile(lat, 99)), 3), "period_ms": round(1e3 / sp["rate"], 3)})
    allv = np.concatenate(lat_all)
    out = {
        "streams": len(specs), "precision": precision, "seconds": seconds, "lines": int(allv.size),
        "throughput_px_s": px / seconds, "p50_ms": float(np.percentile(allv, 50)),
        "p99_ms": float(np.percentile(allv, 99)),
        "p99_ms_by_bands": {str(b): float(np.percentile(np.concatenate(v), 99)) for b, v in sorted(by_b.items())},
        "line_period_ms": [round(1e3 / max(sp["rate"] for sp in specs), 2),
                           round(1e3 / min(sp["rate"] for sp in specs), 2)],
        "streams_p99_below_period": ok_streams, "streams_over_period": over, "pushes": pushes,
        "max_batch": max_batch,
        "engine_error": hs.hsad_status_string(err),
    }
    return out


def run_stress(args, hs, local, world, rank, peaks):
    """32 stored cubes of uneven size scored one by one in CUBE mode (global RX, Sec. 3.3).

    Each cube is drawn on the GPU into one reused buffer (outside the timed region),
    then pushed whole (scored in place) and its scores read into device memory; the
    events bracket push + readback. BF16 and FP32 side by side. Each cube's in-sample
    mean score is checked against the exact B (N-1) / N.
    """
    import numpy as np
    import torch
    from gen import PushbroomScene, stress_cubes
    from gen.device import DeviceScene

    specs = stress_cubes(32)
    if args.stress_cubes:
        specs = specs[:args.stress_cubes]
    if args.cube:  # one cube of a given shape (small cases for profiling)
        Lc, Wc, Bc = (int(v) for v in args.cube.split(","))
        specs = [dict(lines=Lc, width=Wc, bands=Bc, seed=specs[0]["seed"])]
    max_elems = max(s["lines"] * s["width"] * s["bands"] for s in specs)
    max_px = max(s["lines"] * s["width"] for s in specs)
    buf = torch.empty(max_elems, dtype=torch.int16, device=f"cuda:{local}")
    sbuf = torch.empty(max_px, dtype=torch.float32, device=f"cuda:{local}")
    mbuf = torch.empty(max_px, dtype=torch.uint8, device=f"cuda:{local}")
    res = {}
    for prec in ("bf16", "fp32"):
        tot_px, tot_ms, worst, launches, kern = 0, 0.0, 0.0, 0, {}
        for i, sp in enumerate(specs):
            Lc, Wc, Bc = sp["lines"], sp["width"], sp["bands"]
            sc = PushbroomScene(Wc, Bc, seed=sp["seed"] + 1000 * rank)
            x = buf[:Lc * Wc * Bc].view(Lc, Wc, Bc)
            DeviceScene(sc, device=f"cuda:{local}").generate(x, 0, seed=sp["seed"] + 1000 * rank)
            det = hs.Detector(width=Wc, bands=Bc, stats_mode="cube", cube_lines=Lc, precision=prec, gain=sc.gain,
                              offset=sc.offset, result_lines=Lc, device=local)
            det.profile(i == 0)
            stream = torch.cuda.ExternalStream(det.stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n0 = det.kernel_launches
            e0.record(stream)
            rc, first = hs.hsad_push_lines(det.ctx, x, Lc, hs.HSAD_DEVICE)
            assert rc == hs.HSAD_OK, hs.hsad_last_error(det.ctx)
            rc = hs.hsad_scores(det.ctx, first, Lc, sbuf, mbuf, hs.HSAD_DEVICE, -1)
            e1.record(stream)
            e1.synchronize()
            launches += det.kernel_launches - n0
            if i == 0:
                kern = {k: round(ms, 3) for k, (n, ms) in det.profile_totals().items()}
            det.close()
            ms = e0.elapsed_time(e1)
            N = Lc * Wc
            mean = float(sbuf[:N].double().mean())
            worst = max(worst, abs(mean - Bc * (N - 1) / N) / Bc)
            tot_px += N
            tot_ms += ms
        res[prec] = {"value": tot_px * 1e3 / tot_ms, "seconds": tot_ms / 1e3, "cubes": len(specs),
                     "pixels": tot_px, "gpu_launches": launches, "kernels_first_cube_ms": kern,
                     "insample_mean_max_rel_dev": worst}
    del buf
    return res


def main_stress(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle's global RX over 32 cubes of up to "
                              "41M pixels x 448 bands is not a bounded host sample; see the stream workload"}))
        return
    import torch
    import paper_2602_13509_gb300 as hs
    torch.cuda.set_device(local)
    with ClockSampler(local) as clk:
        res = run_stress(args, hs, local, world, rank, load_peaks())
    b = res["bf16"]
    out = {"metric": "pixel-spectra scored/s", "value": b["value"] * world, "unit": "pixel-spectra/s",
           "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": b["seconds"] * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
           "data": "synthetic (drawn on the device)",
           "config": {"workload": f"cube_{args.cube.replace(',', 'x')}" if args.cube else "stress_32_cubes",
                      "cubes": b["cubes"], "stats": "cube (global RX)",
                      "input": "uint16 12-bit DN", "l2": "cubes larger than L2"},
           "fp32_path": res["fp32"], "bf16_path": b, "gpu_launches": b["gpu_launches"], "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(out), flush=True)


# Subsampled kernel RX workload (Sec. 2.2, Table tab:results: 1800 lines x 900 samples x 300
# bands); background subsample size, ridge and kernel width are readings (the paper gives none).
KRX = dict(lines=1800, width=900, bands=300, m=256, ridge=1e-2)


def krx_instr_per_pixel(B, m):
    """FP32-pipe instructions per pixel of the kernel RX scoring kernel as designed: per
    (sample, band) a subtraction, a product and an FMA plus one two-sum per 8 bands (3.75);
    per (output, sample) a float-float multiply-add with a float-float kernel value (12);
    per sample the float-float exponential (reduction and a degree-12 Horner polynomial,
    about 230)."""
    return 3.75 * m * B + 12.0 * m * m + 230.0 * m


def run_krx(args, hs, local, rank, peaks):
    """Subsampled kernel RX of one stored cube (global, every pixel against a random
    background subsample), through hsad_krx, inputs resident in HBM."""
    import numpy as np
    import torch
    from gen import PushbroomScene, subsample_indices
    from gen.device import DeviceScene
    L, W, B, m = KRX["lines"], KRX["width"], KRX["bands"], KRX["m"]
    if args.lines:
        L = args.lines
    n = L * W
    sc = PushbroomScene(W, B, seed=20260213 + 7)
    x = torch.empty((L, W, B), dtype=torch.int16, device=f"cuda:{local}")
    DeviceScene(sc, device=f"cuda:{local}").generate(x, 0, seed=20260213 + 7 + 1000 * rank)
    idx = subsample_indices(n, m, seed=20260213 + 7)
    s = torch.empty(n, dtype=torch.float32, device=f"cuda:{local}")
    mk = torch.empty(n, dtype=torch.uint8, device=f"cuda:{local}")
    stream = torch.cuda.current_stream(local)

    def call():
        rc = hs.hsad_krx(x, n, B, hs.HSAD_U16, idx, 0.0, KRX["ridge"], sc.gain, hs.HSAD_ABS, 0.0, 0, s, mk,
                         stream.cuda_stream, local)
        assert rc == hs.HSAD_OK, hs.hsad_status_string(rc)

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        call()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    acc, cpu = None, None
    if rank == 0 and not args.skip_cpu:
        from oracle import krx as okrx
        host = x.cpu().numpy().view(np.uint16).reshape(n, B)
        t0 = time.perf_counter()
        bg = okrx.krx_background(okrx.calibrate(host[idx], sc.gain, sc.offset), okrx.RBF, 0.0, KRX["ridge"])
        sample = np.random.default_rng(1).choice(n, 2048, replace=False)
        ref = okrx.krx_scores(okrx.calibrate(host[sample], sc.gain, sc.offset), bg)
        secs = time.perf_counter() - t0
        d = s.cpu().numpy()[sample].astype(np.float64)
        e = np.abs(d - ref) / np.maximum(ref, 1.0)
        acc = {"pixels": int(sample.size), "max_rel_err": float(e.max()), "tolerance": 1e-4}
        cpu = {"value": sample.size / secs, "unit": "pixel-spectra/s", "cores": len(os.sched_getaffinity(0)),
               "kind": "oracle", "sample": f"the background statistics (m = {m}) and 2048 random pixels of "
                                           "the cube, the background step counted once as in one cube"}
    mhz = peaks["sm_max_mhz"]
    instr = krx_instr_per_pixel(B, m) * n
    pk = 152 * mhz * 1e6 * 128 / 1e12   # FP32-pipe instructions, T/s
    ach = instr / (ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "Tinstr/s", "frac": ach / pk, "traffic": None,
            "kernel": "krx (whole call: background statistics + per-pixel scoring)",
            "work_per_launch": f"{n} px x (3.75 m B + 12 m^2 + 230 m) FP32-pipe instructions",
            "peak_source": "derived: 152 SMs x %.0f MHz x 128 FP32 lanes" % mhz}
    return {"value": n / (ms / 1e3), "ms": ms, "pixels": n, "accuracy_vs_oracle": acc, "cpu_baseline": cpu,
            "roofline": roof}


def main_krx(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the kernel RX workload's reference is the oracle "
                              "timed in the cpu_baseline of the ours arm"}))
        return
    import torch
    import paper_2602_13509_gb300 as hs
    torch.cuda.set_device(local)
    with ClockSampler(local) as clk:
        r = run_krx(args, hs, local, rank, load_peaks())
    out = {"metric": "pixel-spectra scored/s", "value": r["value"] * world, "unit": "pixel-spectra/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp32 (float-float sums)",
           "data": "synthetic (drawn on the device)",
           "config": {"workload": "krx_1800x900x300", "lines": args.lines or KRX["lines"], "width": KRX["width"],
                      "bands": KRX["bands"], "background_m": KRX["m"], "ridge": KRX["ridge"],
                      "kernel_width": "mean squared distance of distinct background pairs",
                      "l2": "input larger than L2 (%.2f GB)" % (r["pixels"] * KRX["bands"] * 2 / 1e9)},
           "accuracy_vs_oracle": r["accuracy_vs_oracle"], "roofline": r["roofline"],
           "cpu_baseline": r["cpu_baseline"], "gpu_launches": 7 * args.steps, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(out), flush=True)


class _Uncalibrated:
    """Calibration of a front-end workload: none (the scene's gains are per raw band)."""
    gain = None
    offset = None


def make_inputs(wl, rank):
    import numpy as np
    from gen import PushbroomScene, SEED_BASE
    seed = SEED_BASE + (2 if wl["bands"] == 270 else 3) + 1000 * rank
    if wl.get("raw_bands"):
        sc = PushbroomScene(wl["width"], wl["raw_bands"], seed=seed + 7)
        return _Uncalibrated(), sc.lines(0, wl["lines"])  # raw lines
    sc = PushbroomScene(wl["width"], wl["bands"], seed=seed)
    lines = sc.lines(0, wl["lines"])
    return sc, lines


def oracle_lines(wl, lines):
    """The lines the oracle scores: the oracle's own front end of raw lines, else as given."""
    if not wl.get("raw_bands"):
        return lines
    import oracle
    return oracle.frontend(lines, wl["band_first"], wl["band_bin"], wl["bands"])


def run_reference(args, wl, rank, world):
    """The FP64 oracle timed on the host: each step scores one line against all lines before
    it (EXCLUSIVE). Its cost grows with the line index, so the sampled line is the stream
    midpoint (the stream average) unless warm-up + steps lines there would not finish in
    about two minutes; then an earlier line, which overstates the oracle's average rate."""
    if rank != 0:
        return
    T = wl["lines"]
    mid = T // 2
    n_oracle = args.warmup + args.steps
    sc, lines = make_inputs(dict(wl, lines=min(T, 65)), 0)
    lines = oracle_lines(wl, lines)
    # calibrate: the cost of a line against 64 earlier lines, scaled linearly in the index
    _, c64 = oracle_sample(lines, [64 if T > 64 else T - 1], sc.gain, sc.offset)
    budget = 120.0 / max(1, n_oracle)
    t_s = int(min(mid, max(64, 64 * budget / max(c64, 1e-6))))
    sc, lines = make_inputs(dict(wl, lines=min(T, t_s + args.steps + 1)), 0)
    lines = oracle_lines(wl, lines)
    cores = len(os.sched_getaffinity(0))
    for i in range(args.warmup):
        oracle_sample(lines, [t_s - 1 - i], sc.gain, sc.offset)
    px_total, secs = 0, 0.0
    for i in range(args.steps):
        px, s = oracle_sample(lines, [t_s + i], sc.gain, sc.offset)
        px_total += px
        secs += s
    v = px_total / secs
    where = ("the stream midpoint, whose cost equals the stream average" if t_s >= mid else
             f"before the stream midpoint ({mid}) so that {n_oracle} lines finish in minutes: the oracle's "
             f"cost per line grows with the index, so this overstates its stream-average rate about "
             f"{mid / t_s:.1f}x")
    out = {
        "metric": "pixel-spectra scored/s", "value": v, "unit": "pixel-spectra/s", "impl": "reference",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "width": wl["width"], "bands": wl["bands"], "lines": T,
                   "stats": "exclusive", "parallelism": "none (host oracle)"},
        "cpu_baseline": {"value": v, "unit": "pixel-spectra/s", "cores": cores, "kind": "oracle",
                         "sample": f"one line per step (t = {t_s}..{t_s + args.steps - 1}) scored against all "
                                   f"lines before it; {where}"},
        "e2e": {"value": v, "unit": "pixel-spectra/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="precision_1024x448", choices=sorted(WORKLOADS) + ["stress", "krx"])
    ap.add_argument("--stress-cubes", type=int, default=0, help="score only the first k of the 32 cubes")
    ap.add_argument("--cube", default="", help="stress workload: one cube 'lines,width,bands' instead")
    ap.add_argument("--precision", default="fp32", choices=["bf16", "fp16", "fp32"],
                    help="the headline arm (the paper's detector computes in FP32, Sec. 3.4)")
    ap.add_argument("--factor-precision", default="ff", choices=["ff", "fp64"],
                    help="arithmetic of the factor's O(B^3) work: float-float (default) or FP64")
    ap.add_argument("--batch", type=int, default=0, help="lines per internal batch (0 = workload default)")
    ap.add_argument("--factor-every", type=int, default=0,
                    help="factorisation cadence in lines (an extension: statistics up to k-1 lines old); "
                         "0 = every line, the paper's detector")
    ap.add_argument("--lines", type=int, default=0, help="override the stream length (profiling captures)")
    ap.add_argument("--latency-lines", type=int, default=200)
    ap.add_argument("--forget", type=float, default=0.0,
                    help="exponential forgetting factor of the statistics (0 = off)")
    ap.add_argument("--line-gain", action="store_true",
                    help="push every line with its own gain (per-line gain correction)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-other-arm", action="store_true",
                    help="skip the second precision (and the FP64-factor) arms")
    ap.add_argument("--serving-seconds", type=float, default=5.0,
                    help="measured seconds of the 16-stream serving run (0 = skip)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload == "stress":
        return main_stress(args)
    if args.workload == "krx":
        return main_krx(args)
    wl = dict(WORKLOADS[args.workload])
    if args.batch:
        wl["batch"] = args.batch
    if args.lines:
        wl["lines"] = args.lines

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return

    import numpy as np
    import torch
    import paper_2602_13509_gb300 as hs

    torch.cuda.set_device(local)
    host_cpus = bind_near_gpu(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    peaks = load_peaks()
    sc, lines = make_inputs(wl, rank)
    T, W, B = wl["lines"], wl["width"], wl["bands"]
    x_dev = torch.from_numpy(lines.view(np.int16)).to(f"cuda:{local}")
    x_host = torch.from_numpy(lines.view(np.int16)).pin_memory()
    s_dev = torch.empty((T, W), dtype=torch.float32, device=f"cuda:{local}")
    m_dev = torch.empty((T, W), dtype=torch.uint8, device=f"cuda:{local}")
    s_host = torch.empty((T, W), dtype=torch.float32).pin_memory()
    m_host = torch.empty((T, W), dtype=torch.uint8).pin_memory()

    def detector(prec, factor="ff"):
        return hs.Detector(width=W, bands=B, stats_mode="exclusive", precision=prec, factor_precision=factor,
                           gain=sc.gain,
                           offset=sc.offset, max_batch_lines=wl["batch"], result_lines=T, device=local,
                           raw_bands=wl.get("raw_bands", 0), band_first=wl.get("band_first", 0),
                           band_bin=wl.get("band_bin", 1), factor_every=args.factor_every, forget=args.forget)

    # per-line gain correction (Sec. 3.2): every line pushed with its own gain
    line_gain = (np.random.default_rng(7).uniform(0.8, 1.25, size=T).astype(np.float32)
                 if args.line_gain else None)

    def push(det, x, mem):
        if line_gain is None:
            return hs.hsad_push_lines(det.ctx, x, T, mem)
        return hs.hsad_push_lines_gain(det.ctx, x, line_gain, T, mem)

    def step(det, host=False):
        det.reset()
        if host:
            rc, first = push(det, x_host, hs.HSAD_HOST)
            assert rc == hs.HSAD_OK, hs.hsad_last_error(det.ctx)
            rc = hs.hsad_scores(det.ctx, first, T, s_host, m_host, hs.HSAD_HOST, -1)
        else:
            rc, first = push(det, x_dev, hs.HSAD_DEVICE)
            assert rc == hs.HSAD_OK, hs.hsad_last_error(det.ctx)
            rc = hs.hsad_scores(det.ctx, first, T, s_dev, m_dev, hs.HSAD_DEVICE, -1)
        assert rc in (hs.HSAD_OK, hs.HSAD_E_NOT_READY), hs.hsad_status_string(rc)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(det, host=False, clocks=None):
        for _ in range(args.warmup):
            step(det, host)
        stream = torch.cuda.ExternalStream(det.stream)
        barrier()
        n0 = det.kernel_launches
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step(det, host)
        e1.record(stream)
        e1.synchronize()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, f"cuda:{local}")
        return ms, det.kernel_launches - n0

    px_step = T * W
    other = "bf16" if args.precision != "bf16" else "fp32"

    def measure(prec, factor="ff", clocks=False):
        """Device-resident throughput of one arm, then per-kernel CUDA-event times (separate
        pass) and the scores of the accuracy sample line. Leaves the detector open."""
        det = detector(prec, factor)
        form = det.whitening_form
        tcw = det.whitening_tensor_cores
        if clocks:
            with ClockSampler(local) as clk:
                ms, launches = timed(det)
            clk_summary = clk.summary()
        else:
            ms, launches = timed(det)
            clk_summary = None
        # per-kernel times, CUDA events on the library's stream (separate pass)
        det.profile(True)
        det.profile_reset()
        for _ in range(prof_steps):
            step(det)
        prof = det.profile_totals()
        det.profile(False)
        sample = s_dev[t_acc].cpu().numpy().copy(), m_dev[t_acc].cpu().numpy().copy()
        return det, dict(value=weak_value(px_step, world, ms), ms=ms, launches=launches, form=form, tc=tcw, prof=prof,
                         sample=sample, clocks=clk_summary)

    prof_steps = 2
    t_acc = T // 2   # the accuracy sample: scored by the oracle once, compared with every arm
    det, head = measure(args.precision, args.factor_precision, clocks=True)
    ms, launches, form, prof = head["ms"], head["launches"], head["form"], head["prof"]
    tcw = head["tc"]
    value = head["value"]
    per_kernel = {k: {"launches_per_step": n / prof_steps, "ms_per_step": t / prof_steps}
                  for k, (n, t) in prof.items()}
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None

    lat = {}
    if rank == 0 and args.latency_lines > 0:
        det.reset()
        warm = (B + 1 + W - 1) // W + 2 + 64
        hs.hsad_push_lines(det.ctx, x_host[:warm], warm, hs.HSAD_HOST)
        det.synchronize()
        one_s = torch.empty((1, W), dtype=torch.float32).pin_memory()
        one_m = torch.empty((1, W), dtype=torch.uint8).pin_memory()
        # lines arrive at the sensor's rate (249 lines/s, Sec. 3.2); latency = scores on
        # the host minus the line's scheduled arrival
        period = 1.0 / 249.0
        n_lat = min(T - warm, args.latency_lines)
        samples = []
        t_start = time.perf_counter() + 0.01
        for k in range(n_lat):
            t_sched = t_start + k * period
            while time.perf_counter() < t_sched:
                pass
            rc, first = hs.hsad_push_lines(det.ctx, x_host[warm + k:warm + k + 1], 1, hs.HSAD_HOST)
            rc = hs.hsad_scores(det.ctx, first, 1, one_s, one_m, hs.HSAD_HOST, -1)
            samples.append((time.perf_counter() - t_sched) * 1e3)
        # back to back (no pacing): each line also waits for the previous line's factorisation
        b2b = []
        for k in range(min(64, T - warm - n_lat)):
            t0 = time.perf_counter()
            rc, first = hs.hsad_push_lines(det.ctx, x_host[warm + n_lat + k:warm + n_lat + k + 1], 1, hs.HSAD_HOST)
            rc = hs.hsad_scores(det.ctx, first, 1, one_s, one_m, hs.HSAD_HOST, -1)
            b2b.append((time.perf_counter() - t0) * 1e3)
        samples.sort()
        b2b.sort()
        lat = {"p50_ms": samples[len(samples) // 2], "p99_ms": samples[min(len(samples) - 1, int(0.99 * len(samples)))],
               "lines": len(samples), "line_period_ms": 1e3 * period,
               "back_to_back_p50_ms": b2b[len(b2b) // 2] if b2b else None,
               "what": "one stream, lines pushed from host memory at 249 lines/s; scheduled arrival to "
                       "scores on the host"}

    serving = None
    if rank == 0 and args.serving_seconds > 0:
        serving = {p: run_serving(hs, local, p, args.serving_seconds, 1.0) for p in ("bf16", "fp32")}

    # transmit encoding (Sec. 3.4) of the step's last full ring of scores, through the
    # public API into device memory (a full call: launches, copy stream sync included)
    tx = None
    if rank == 0:
        step(det)  # the latency leg above restarted the stream: score lines 0 .. T-1 again
        n_tx, first_tx = T, 0
        codes = torch.empty((n_tx, W), dtype=torch.int16, device=f"cuda:{local}")
        for _ in range(3):
            hs.hsad_scores_tx(det.ctx, first_tx, n_tx, codes, hs.HSAD_DEVICE, -1)
        t0 = time.perf_counter()
        reps = 20
        for _ in range(reps):
            rc_tx, _ = hs.hsad_scores_tx(det.ctx, first_tx, n_tx, codes, hs.HSAD_DEVICE, -1)
        tx_ms = (time.perf_counter() - t0) * 1e3 / reps
        assert rc_tx in (hs.HSAD_OK, hs.HSAD_E_NOT_READY), hs.hsad_status_string(rc_tx)
        tx = {"lines": n_tx, "ms_per_call": tx_ms, "status": hs.hsad_status_string(rc_tx),
              "bytes_per_pixel": 6, "what": "hsad_scores_tx: block maximum + binary16(sqrt(delta/max)) codes, "
                                            "device output, host-timed API call"}

    # end to end through the public API from pinned host memory
    e2e_ms, _ = timed(det, host=True)
    e2e = {"value": px_step * world / (e2e_ms / 1e3), "unit": "pixel-spectra/s",
           "h2d_bytes_per_step": int(x_host.numel() * 2), "d2h_bytes_per_step": int(T * W * 5)}
    det.close()

    # the other precision on the same workload and step count, and the FP32 path with the
    # FP64 factor (precision forms side by side)
    arms = {}
    if not args.skip_other_arm:
        d2, arm = measure(other, args.factor_precision)
        e2_ms, _ = timed(d2, host=True)
        d2.close()
        arm["e2e"] = {"value": px_step * world / (e2_ms / 1e3), "unit": "pixel-spectra/s"}
        arms[other] = arm
        if args.precision == "fp32" and args.factor_precision == "ff":
            d3, arm3 = measure("fp32", "fp64")
            d3.close()
            arms["fp32_fp64_factor"] = arm3

    mhz = peaks["sm_max_mhz"]
    head_roofs = kernel_rooflines(prof, prof_steps, T, W, B, form, args.precision, args.factor_every, peaks, mhz,
                                  tcw, args.workload)
    roof = dict(head_roofs[dom]) if dom in head_roofs else None

    cpu, ref_line = None, None
    if rank == 0 and not args.skip_cpu:
        px, secs, ref_line = oracle_sample_scores(oracle_lines(wl, lines[:t_acc + 1]), t_acc, sc.gain, sc.offset)
        cpu = {"value": px / secs, "unit": "pixel-spectra/s", "cores": len(os.sched_getaffinity(0)),
               "kind": "oracle", "sample": f"line {t_acc} of the stream ({W} pixels) scored against lines "
                                           f"0..{t_acc - 1}; its cost equals the stream average"}

    def accuracy(arm, prec):
        if ref_line is None:
            return None
        s_, m_ = arm["sample"]
        return accuracy_vs_oracle(s_, m_, ref_line, B, prec, t_acc)

    def arm_json(arm, prec):
        pk = {k: {"launches_per_step": n / prof_steps, "ms_per_step": t / prof_steps}
              for k, (n, t) in arm["prof"].items()}
        return {"value": arm["value"], "unit": "pixel-spectra/s", "ms_per_step": arm["ms"], "dtype": prec,
                "gpu_launches": arm["launches"], "e2e": arm.get("e2e"),
                "whitening": whitening_label(arm["form"], arm["tc"]),
                "accuracy_vs_oracle": accuracy(arm, prec), "kernels": pk,
                "rooflines": kernel_rooflines(arm["prof"], prof_steps, T, W, B, arm["form"], prec,
                                              args.factor_every, peaks, mhz, arm["tc"], args.workload)}

    out = {
        "metric": "pixel-spectra scored/s", "value": value, "unit": "pixel-spectra/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": args.workload, "width": W, "bands": B, "lines": T, "stats": "exclusive",
                   "input": "uint16 12-bit DN", "batch_lines": wl["batch"],
                   "whitening": whitening_label(form, tcw),
                   "factor": "FP64" if args.factor_precision == "fp64" else "float-float",
                   **({"factor_every": args.factor_every} if args.factor_every > 1 else {}),
                   **({"line_gain": "per-line gains U[0.8, 1.25] (hsad_push_lines_gain)"} if args.line_gain else {}),
                   **({"forget": args.forget} if 0.0 < args.forget < 1.0 else {}),
                   **({"front_end": {"raw_bands": wl["raw_bands"], "band_first": wl["band_first"],
                                     "band_bin": wl["band_bin"]}} if wl.get("raw_bands") else {}),
                   "parallelism": f"replicas x{world} (independent streams)" if world > 1 else "single stream",
                   "l2": "inputs larger than L2 (%.2f GB per step)" % (x_dev.numel() * 2 / 1e9),
                   "host": host_cpus},
        "accuracy_vs_oracle": accuracy(head, args.precision),
        "latency": lat, "e2e": e2e, "gpu_launches": launches,
        **{f"{k}_path": arm_json(a, "fp32" if k == "fp32_fp64_factor" else k) for k, a in arms.items()},
        "roofline": roof, "rooflines": head_roofs, "kernels": per_kernel, "cpu_baseline": cpu,
        "clocks": head["clocks"], "serving": serving, "tx_encode": tx,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
