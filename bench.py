#!/usr/bin/env python
"""Throughput of the two-stage hierarchical matched-filter hot path on GB300.

Workload (one step): two detectors, 512 s of strain at 2048 Hz with coloured
Gaussian noise, 20 sine-Gaussian glitches and 50 TaylorF2 injections per
segment; stage 1 filters a 2,000-template coarse bank on the data decimated to
512 Hz (N = 2^18, threshold 3.5), coincidences with 101 time shifts select
coarse templates with network SNR >= 7, stage 2 filters the union of their
neighbourhoods (match >= 0.9) in a 20,000-template fine bank at 2048 Hz
(N = 2^20, threshold 4).  Everything from the strain to the trigger lists runs
in libmf's kernels.

Metric: template-seconds (one template over one second of one detector's
data) filtered per second.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "template-seconds filtered/s on 1 GB300 at SNR err<=1e-3; % HBM roofline"
UNIT = "template-seconds/s"
WORKLOAD = ("two-stage hierarchical search: 2 det x 512 s @ 2048 Hz, coarse 2000 @ 512 Hz (N=2^18), "
            "fine 20000 @ 2048 Hz (N=2^20) on the nbhd union")
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# names of the two filter kernels per plan implementation (mf_plan_stats.impl)
KERNEL_NAMES = {2: ("k_cols", "k_rows")}


def measured_traffic(kernel, series_per_launch):
    """DRAM bytes per launch of `kernel` from the committed ncu summaries (lines
    'bench-traffic: <kernel> series=<s> dram_bytes=<b>'), scaled from the captured
    launch's s series to this launch's series (the traffic of these kernels grows in
    proportion to the series they process), or None."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    name = kernel.split(" ")[0].replace(" ", "")
    for fn in sorted(os.listdir(d)):
        if not fn.endswith((".md", ".txt")):
            continue
        with open(os.path.join(d, fn)) as fh:
            for line in fh:
                if line.startswith("bench-traffic:"):
                    f = line.split()
                    if f[1] == name:
                        series = int(f[2].split("=")[1])
                        return int(f[3].split("=")[1]) * float(series_per_launch) / series
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--small", action="store_true", help="32 s scaled-down workload (quick checks only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU baseline sample")
    ap.add_argument("--kernel-case", type=int, default=0, metavar="LOG2N",
                    help="instead of the benchmark, run two mf_filter calls on a 2-detector plan with N = 2^LOG2N "
                         "(a small, fixed case for profiler captures) and exit")
    ap.add_argument("--kernel-templates", type=int, default=16)
    return ap.parse_args()


def kernel_case(lg, n_tmpl):
    """Two filter calls of a 2-detector, n_tmpl-template plan at N = 2^lg (TaylorF2 bank,
    coloured noise); used as the fixed workload of profiler captures."""
    import torch

    import synth
    from paper_2309_00019_gb300 import _build, mf

    if not os.path.exists(mf.LIB_PATH):
        _build.build()
    n = 1 << lg
    fs = 2048.0 if lg >= 19 else 512.0
    rng = np.random.default_rng(0)
    dev = torch.device("cuda:0")
    m1, m2 = synth.sample_bank_uniform_masses(rng, n_tmpl, 1.4, 10.0)
    bank = synth.taylorf2_torch(n, fs, m1, m2, 30.0, dev)
    fd = np.stack([synth.coloured_noise_fd(rng, n, fs) for _ in range(2)]).astype(np.complex64)
    p = mf.Plan(fs, n, 2, 30.0, fs / 2, 4.0, int(fs))
    p.set_psd(synth.psd_bins(n, fs))
    p.load_bank(bank)
    d = torch.from_numpy(fd).to(dev)
    for _ in range(2):
        p.filter(d)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": lg, "templates": n_tmpl, "triggers": p.triggers()[1],
                      "impl": p.stats()["impl"], "batch": p.stats()["batch"]}))
    p.close()
    return 0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                    power.append(float(f[3]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# CPU oracle timing (reported baseline; also the --impl reference arm)
# ---------------------------------------------------------------------------

def oracle_sample_rate(cfg, budget_s, n_each=None):
    """Time the FP64 oracle, as it stands, filtering coarse templates at stage 1
    and fine templates at stage 2 (both detectors), alternating one template of
    each, until the budget is spent.  Returns (td-s/s, cores, description)."""
    from oracle import mf_oracle as O

    s2 = O.strain_to_fd(cfg.strain, cfg.fs2)
    s1 = O.decimate_fd(s2, cfg.n1)
    t0 = time.perf_counter()
    td = 0.0
    k = 0
    while True:
        cb = cfg.coarse_bank([k % len(cfg.coarse_m1)], dtype=np.complex128)
        O.filter_bank(s1, cb, cfg.psd1, cfg.n1, cfg.fs1, cfg.f_low, cfg.fs1 / 2, cfg.thr1, cfg.window1)
        fb = cfg.fine_bank([k % len(cfg.fine_m1)], dtype=np.complex128)
        O.filter_bank(s2, fb, cfg.psd2, cfg.n2, cfg.fs2, cfg.f_low, cfg.fs2 / 2, cfg.thr2, cfg.window2)
        td += 2 * cfg.n1 / cfg.fs1 + 2 * cfg.n2 / cfg.fs2
        k += 1
        el = time.perf_counter() - t0
        if (n_each is not None and k >= n_each) or (n_each is None and el >= budget_s):
            break
    desc = (f"oracle filter_bank (numpy FP64, 1 thread) on {k} coarse templates at 512 Hz and {k} fine "
            f"templates at 2048 Hz, 2 detectors, 512 s segment, {el:.1f} s")
    return td / el, 1, desc, el


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

def dist_setup(args):
    from paper_2309_00019_gb300.multi import rank_env
    return rank_env()


def reference_arm(args, rank, world):
    import synth

    if rank != 0:
        return 0
    cfg = synth.make_config2(seed=1, small=args.small)
    for _ in range(args.warmup):
        oracle_sample_rate(cfg, 0, n_each=1)
    times, tds = [], []
    for _ in range(args.steps):
        rate, cores, desc, el = oracle_sample_rate(cfg, 0, n_each=2)
        times.append(el)
        tds.append(rate * el)
    value = sum(tds) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if not args.small else "scaled-down 32 s hierarchy (check run)",
                   "l2": "n/a (CPU)", "parallelism": "1 segment on the host cores (rank 0 only)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"per step: {desc}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.kernel_case:
        return kernel_case(args.kernel_case, args.kernel_templates)
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch

    import synth
    from paper_2309_00019_gb300 import _build, mf
    from paper_2309_00019_gb300.hierarchy import HierParams, Hierarchy
    from paper_2309_00019_gb300.multi import reduce_timing, segment_seed

    if not os.path.exists(mf.LIB_PATH):
        _build.build()
    mf.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    cfg = synth.make_config2(seed=segment_seed(1, rank), small=args.small)
    hp = HierParams.from_config(cfg)
    h = Hierarchy(hp, cfg.psd1, cfg.psd2, len(cfg.coarse_m1), len(cfg.fine_m1), cfg.nbhd_ptr, cfg.nbhd_idx,
                  device=dev)
    for r0, rows in synth.taylorf2_chunks_torch(cfg.n1, cfg.fs1, cfg.coarse_m1, cfg.coarse_m2, cfg.f_low, dev,
                                                chunk=256, ld=h.ld1):
        h.set_bank_rows(1, r0, rows)
    for r0, rows in synth.taylorf2_chunks_torch(cfg.n2, cfg.fs2, cfg.fine_m1, cfg.fine_m2, cfg.f_low, dev,
                                                chunk=64, ld=h.ld2):
        h.set_bank_rows(2, r0, rows)
    torch.cuda.empty_cache()
    h.strain.copy_(torch.from_numpy(cfg.strain))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # 512 MB > L2 (126 MB)
    st = h.stream

    # warm-up
    for _ in range(max(args.warmup, 0)):
        h.run()
    torch.cuda.synchronize()

    # timed region: per-step CUDA events on the plans' stream, L2 flushed between steps
    for p in (h.p1, h.p2):
        p.stats(reset=True)
        p.profile(True)
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    td_total = 0.0
    unions = []
    wall0 = time.perf_counter()
    for i in range(args.steps):
        with torch.cuda.stream(st):
            flush.zero_()
            ev[i][0].record(st)
        h.run()
        with torch.cuda.stream(st):
            ev[i][1].record(st)
        td_total += h.td_seconds()
        unions.append(h.n_union)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    s1, s2 = h.p1.stats(reset=True), h.p2.stats(reset=True)
    for p in (h.p1, h.p2):
        p.profile(False)
    t_dev = sum(step_ms) / 1e3
    if dist is not None:
        t_max, td_all = reduce_timing(dist, t_dev, td_total, dev)
    else:
        t_max, td_all = t_dev, td_total
    value = td_all / t_max

    # dominant kernel (profiled launches of the timed region): ALU roofline and HBM view
    kinds = []
    for stage, s, n in (("stage1", s1, hp.n1), ("stage2", s2, hp.n2)):
        lg = int(round(math.log2(n)))
        n1s, n2s = 1 << ((lg + 1) // 2), 1 << (lg // 2)
        names = KERNEL_NAMES.get(s["impl"], ("pass1", "pass2"))
        nb = n // 2 + 1
        for k, sub, nm in (("pass1", n1s, names[0]), ("pass2", n2s, names[1])):
            if s[f"{k}_launches"] > 0:
                kinds.append(dict(kernel=f"{nm}<{n1s},{n2s}> ({stage})", ms=s[f"{k}_ms"],
                                  launches=s[f"{k}_launches"], series=s[f"{k}_series"],
                                  flops_series=5.0 * n * math.log2(sub), n=n,
                                  tmpl_bytes_series=(nb * 8 / hp.n_det) if k == "pass1" else 0.0))
    dom = max(kinds, key=lambda d: d["ms"]) if kinds else None
    roof = None
    hbm_gbs, hbm_kind = peaks()
    alu_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    try:  # measured FP32 FMA throughput (context for the derived peak)
        alu_probe = mf.fma_probe()
    except Exception:
        alu_probe = None
    klist = []
    for d in kinds:
        per_ms = d["ms"] / d["launches"]
        spl = d["series"] / d["launches"]
        klist.append({"kernel": d["kernel"], "launches": d["launches"], "ms_total": d["ms"],
                      "per_launch_ms": per_ms, "series_per_launch": spl,
                      "alu_tflops": spl * d["flops_series"] / (per_ms * 1e-3) / 1e12,
                      "template_gbs": spl * d["tmpl_bytes_series"] / (per_ms * 1e-3) / 1e9})
    if dom is not None:
        per_launch_ms = dom["ms"] / dom["launches"]
        spl = dom["series"] / dom["launches"]
        achieved = spl * dom["flops_series"] / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": measured_traffic(dom["kernel"], spl),
                "kernel": dom["kernel"], "per_launch_ms": per_launch_ms, "series_per_launch": spl,
                "flops_per_series": dom["flops_series"],
                "flop_convention": "5 N log2(M) per series for an N-point transform built from M-point sub-FFTs",
                "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (derived, not measured)",
                "alu_probe_tflops": alu_probe,
                "frac_of_probe": achieved / alu_probe if alu_probe else None,
                "kernels": klist}
    # whole-step HBM view: template bytes the step must stream / step time
    step_bytes = (len(cfg.coarse_m1) * (hp.n1 // 2 + 1) + statistics.mean(unions) * (hp.n2 // 2 + 1)) * 8
    step_hbm = step_bytes / (t_dev / args.steps) / 1e9

    # end to end through the public API from pinned host strain, triggers read back
    e2e = None
    if not args.no_e2e:
        pinned = torch.from_numpy(cfg.strain).pin_memory()
        h.run_host(pinned)
        torch.cuda.synchronize()
        te, td_e, d2h = [], 0.0, 0
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            trig2, co = h.run_host(pinned)
            torch.cuda.synchronize()
            te.append(time.perf_counter() - t0)
            td_e += h.td_seconds()
            d2h += trig2.nbytes + co.nbytes + 16
        e_val = td_e / sum(te)
        if dist is not None:
            t_e, td_e_all = reduce_timing(dist, sum(te), td_e, dev)
            e_val = td_e_all / t_e
        e2e = {"value": e_val, "unit": UNIT, "h2d_bytes_per_step": int(cfg.strain.nbytes),
               "d2h_bytes_per_step": int(d2h / args.steps)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, desc, _ = oracle_sample_rate(cfg, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if not args.small else "scaled-down 32 s hierarchy (check run)",
                       "union_templates": int(statistics.mean(unions)),
                       "td_seconds_per_step": td_total / args.steps,
                       "l2": "512 MB buffer written between timed steps; banks (1 GB + 84 GB) streamed from HBM",
                       "parallelism": f"{world} independent segments (one per GPU)"},
            "roofline": roof,
            "hbm_step": {"template_bytes_per_step": step_bytes, "achieved_gbs": step_hbm, "peak_gbs": hbm_gbs,
                         "frac": step_hbm / hbm_gbs, "peak_kind": hbm_kind},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(s1["launches"] + s2["launches"]),
            "clocks": clk,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
