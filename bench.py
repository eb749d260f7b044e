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
data) filtered per second at SNR error <= 1e-3.  Stage 2 runs with the FP16
pass-1 -> pass-2 intermediate and the tensor-core row pass by default
(--intermediate f32 for the FP32 ALU row pass).  Prints one JSON line (rank 0).

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
            "fine 20000 @ 2048 Hz (N=2^20) on the union of exact-match (>= 0.9) neighbourhoods")
FP32_LANES_PER_SM = 128
# names of the two filter kernels per plan implementation (mf_plan_stats.impl)
# k_cols_h16 / k_cols_h16x2: k_cols with FP16 / FP16-pair output; k_rows_tc2: the split-product row pass
KERNEL_NAMES = {2: ("k_cols", "k_rows"), 3: ("k_cols_h16", "k_rows_tc"), 4: ("k_cols_h16x2", "k_rows_tc2")}
# the timed steps time every PROFILE_STRIDE-th launch pair of the filter kernels: the events between the two
# passes of a timed pair keep the second kernel from launching early, so the others run undisturbed
PROFILE_STRIDE = 8


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
    ap.add_argument("--workload", choices=["hierarchy", "uneven"], default="hierarchy",
                    help="hierarchy (default): the two-stage search step; uneven: 20,000 templates of uneven "
                         "duration in 4/16/64/256 s length classes over 2 x 4096 s, one fused work queue per pass "
                         "(--impl reference times the default workload's oracle)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU baseline sample")
    ap.add_argument("--kernel-case", type=int, default=0, metavar="LOG2N",
                    help="instead of the benchmark, run two mf_filter calls on a 2-detector plan with N = 2^LOG2N "
                         "(a small, fixed case for profiler captures) and exit")
    ap.add_argument("--kernel-templates", type=int, default=16)
    ap.add_argument("--intermediate", choices=["f32", "f16", "f16x2"], default="f16",
                    help="pass-1 -> pass-2 intermediate of the N = 2^20 (stage-2) filter: f16 (default; tensor-core "
                         "row pass, SNR within 1e-3 of the FP64 oracle, the metric's bar), f16x2 (FP16 pairs and "
                         "split tensor-core products, FP32-level SNR) or f32 (ALU row pass, SNR within 1e-5)")
    return ap.parse_args()


def kernel_case(lg, n_tmpl, inter="f16"):
    """Two filter calls of a 2-detector, n_tmpl-template plan at N = 2^lg (TaylorF2 bank,
    coloured noise); used as the fixed workload of profiler captures.  Prints the
    per-launch times of the two passes of the second call (CUDA events)."""
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
    if inter != "f32" and lg == 20:
        p.set_intermediate(mf.MF_F16 if inter == "f16" else mf.MF_F16X2)
    d = torch.from_numpy(fd).to(dev)
    p.filter(d)
    torch.cuda.synchronize()
    p.stats(reset=True)
    p.profile(True)
    p.filter(d)
    torch.cuda.synchronize()
    st = p.stats(reset=True)
    p.profile(False)
    L = max(st["pass1_launches"], 1)
    print(json.dumps({"kernel_case": lg, "templates": n_tmpl, "triggers": p.triggers()[1], "impl": st["impl"],
                      "batch": st["batch"], "launches": st["pass1_launches"],
                      "pass1_ms_per_launch": st["pass1_ms"] / L, "pass2_ms_per_launch": st["pass2_ms"] / L,
                      "series_per_launch": st["pass1_series"] / L,
                      "us_per_series": 1e3 * (st["pass1_ms"] + st["pass2_ms"]) / max(st["pass1_series"], 1)}))
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
# CPU oracle timing (reported baseline; also the --impl reference arm): the
# oracle as it stands, one process per host core, each filtering its own
# templates (the oracle's numpy FFTs are single-threaded)
# ---------------------------------------------------------------------------

_POOL = {}


def _pool_init(cfg):
    from oracle import mf_oracle as O

    s2 = O.strain_to_fd(cfg.strain, cfg.fs2)
    _POOL.update(cfg=cfg, s2=s2, s1=O.decimate_fd(s2, cfg.n1))


def _pool_work(job):
    """One worker: wait for the common start time, then filter one coarse template
    at stage 1 and one fine template at stage 2 (both detectors) at a time, from
    template k0 on, until `budget` seconds have passed (or n_each pairs are done).
    Returns (template-seconds, pairs, end time)."""
    from oracle import mf_oracle as O

    t_go, budget, n_each, k0 = job
    cfg, s1, s2 = _POOL["cfg"], _POOL["s1"], _POOL["s2"]
    while time.time() < t_go:
        time.sleep(0.001)
    td, k = 0.0, 0
    while True:
        i = k0 + k
        cb = cfg.coarse_bank([i % len(cfg.coarse_m1)], dtype=np.complex128)
        O.filter_bank(s1, cb, cfg.psd1, cfg.n1, cfg.fs1, cfg.f_low, cfg.fs1 / 2, cfg.thr1, cfg.window1)
        fb = cfg.fine_bank([i % len(cfg.fine_m1)], dtype=np.complex128)
        O.filter_bank(s2, fb, cfg.psd2, cfg.n2, cfg.fs2, cfg.f_low, cfg.fs2 / 2, cfg.thr2, cfg.window2)
        td += 2 * cfg.n1 / cfg.fs1 + 2 * cfg.n2 / cfg.fs2
        k += 1
        if (n_each is not None and k >= n_each) or (n_each is None and time.time() - t_go >= budget):
            break
    return td, k, time.time()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                             timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _pool_init_uneven(c, xh, n):
    _POOL.update(c=c, xh=xh, n=n)


def _pool_work_uneven(job):
    """One worker of the uneven-length workload: from template k0 on (strided over the bank, so every length
    class is sampled), the oracle's segmented search of the whole stream with one template, both detectors,
    at the GPU run's segment length; as _pool_work otherwise."""
    import synth
    from oracle import mf_oracle as O

    t_go, budget, n_each, k0 = job
    c, xh, n = _POOL["c"], _POOL["xh"], _POOL["n"]
    psd = synth.psd_bins(n, c.fs)
    while time.time() < t_go:
        time.sleep(0.001)
    td, k = 0.0, 0
    while True:
        i = (k0 + 4099 * k) % len(c.m1)
        ci = int(c.cls[i])
        bank = synth.taylorf2(n, c.fs, c.m1[i], c.m2[i], c.f_low)[None, :]
        O.segmented_filter(xh, c.fs, psd, c.f_low, c.fs / 2, bank, n, int(c.class_len[ci] * c.fs), c.thr, c.window)
        td += 2 * c.n_samples / c.fs
        k += 1
        if (n_each is not None and k >= n_each) or (n_each is None and time.time() - t_go >= budget):
            break
    return td, k, time.time()


class OraclePool:
    """A spawn-started process pool (safe after the GPU is initialised), one
    worker per host core, holding the workload's inputs (init / work: the
    workload's initialiser and sample function)."""

    def __init__(self, cfg, workers=None, init=_pool_init, work=_pool_work, initargs=None):
        import multiprocessing as mp

        self.n = workers or host_cores()
        self.work = work
        self.pool = mp.get_context("spawn").Pool(self.n, initializer=init,
                                                 initargs=initargs if initargs is not None else (cfg,))
        self.pool.map(work, [(0.0, 0.0, 1, 0)] * self.n)  # workers up, imports and first FFTs done
        self.k0 = 0

    def run(self, budget_s=0.0, n_each=None, slack_s=0.5):
        """All workers start together; returns (td-s/s, pairs, wall seconds)."""
        t_go = time.time() + slack_s
        jobs = [(t_go, budget_s, n_each, self.k0 + 7919 * w) for w in range(self.n)]
        self.k0 += 1
        res = self.pool.map(self.work, jobs)
        td = sum(r[0] for r in res)
        el = max(r[2] for r in res) - t_go
        return td / el, sum(r[1] for r in res), el

    def close(self):
        self.pool.terminate()
        self.pool.join()


def oracle_sample_rate(cfg, budget_s):
    """The FP64 oracle, as it stands, on every host core for about budget_s."""
    pool = OraclePool(cfg)
    try:
        rate, pairs, el = pool.run(budget_s)
    finally:
        pool.close()
    desc = (f"oracle filter_bank (numpy FP64) in {pool.n} processes, one per host core: {pairs} coarse templates "
            f"at 512 Hz and {pairs} fine templates at 2048 Hz, 2 detectors, 512 s segment, {el:.1f} s; "
            f"CPU {cpu_model()}")
    return rate, pool.n, desc, el


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
    pool = OraclePool(cfg)
    for _ in range(args.warmup):
        pool.run(n_each=1)
    times, tds = [], []
    for _ in range(args.steps):
        rate, pairs, el = pool.run(n_each=1)
        times.append(el)
        tds.append(rate * el)
    pool.close()
    cores = pool.n
    value = sum(tds) / sum(times)
    desc = (f"oracle filter_bank (numpy FP64) in {cores} processes, one per host core, each filtering one coarse "
            f"template at 512 Hz and one fine template at 2048 Hz (2 detectors, 512 s segment); CPU {cpu_model()}")
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


WORKLOAD_UNEVEN = ("uneven-length bank: 20000 TaylorF2 templates (chirp mass 1.2-10, 2PN durations 2.5-91 s "
                   "from 25 Hz) in 4/16/64/256 s length classes, 2 det x 4096 s @ 2048 Hz in overlapping segments "
                   "of one autotuned length for all classes, one fused work queue over all classes per pass")


def uneven_main(args, rank, world, local):
    """The uneven-length workload: each step is one pass of mf_batch_run(MF_RUN_FUSED) over the stream (segment
    spectra, the fused filter's launch pairs over every class's series, trigger compaction); the same JSON
    line as the default workload.  The fused launch pairs report their CUDA-event times on the first class's
    plan (mf_profile), which gives the roofline object."""
    import torch

    import synth
    from paper_2309_00019_gb300 import _build, mf
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
    c = synth.make_config3(seed=segment_seed(3, rank))
    x = c.strain(dev)
    st = torch.cuda.Stream(device=dev)
    b = mf.Batch(c.fs, 2, c.n_samples, c.f_low, c.fs / 2, c.thr, c.window, c.class_len, stream=st.cuda_stream)
    b.set_psd(c.psd(c.n_fd), c.n_fd)
    n_cls = len(c.class_len)
    n_tmpl = [len(c.class_ids(i)) for i in range(n_cls)]
    b.autotune(n_tmpl, fused=True)  # set-up, untimed
    plans = [b.plan(ci) for ci in range(n_cls)]
    for ci, p in enumerate(plans):
        ids = c.class_ids(ci)
        p.bank_reserve(len(ids))
        p.bank_generate_taylorf2(0, c.m1[ids], c.m2[ids], c.f_low)
        if args.intermediate != "f32":
            p.set_intermediate(mf.MF_F16 if args.intermediate == "f16" else mf.MF_F16X2)
    seg = [b.segment(ci) for ci in range(n_cls)]
    n = seg[0]["n"]
    td_step = sum(n_tmpl) * 2 * c.n_samples / c.fs
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    mode = mf.MF_RUN_FUSED
    for _ in range(max(args.warmup, 0)):
        b.run(x, mode=mode)
    torch.cuda.synchronize()
    for p in plans:
        p.stats(reset=True)
    plans[0].profile(PROFILE_STRIDE)
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for i in range(args.steps):
        with torch.cuda.stream(st):
            flush.zero_()
            ev[i][0].record(st)
        b.run(x, mode=mode)
        with torch.cuda.stream(st):
            ev[i][1].record(st)
        plans[0].stats()  # reads this step's launch-pair events (up to 4096 per read)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b_) for a, b_ in ev]
    sts = [p.stats(reset=True) for p in plans]
    plans[0].profile(False)
    t_dev = sum(step_ms) / 1e3
    td_total = td_step * args.steps
    if dist is not None:
        t_max, td_all = reduce_timing(dist, t_dev, td_total, dev)
    else:
        t_max, td_all = t_dev, td_total
    value = td_all / t_max

    hbm_gbs, hbm_kind = peaks()
    s0 = sts[0]
    lg = int(round(math.log2(n)))
    n1s, n2s = 1 << ((lg + 1) // 2), 1 << (lg // 2)
    names = KERNEL_NAMES.get(s0["impl"], ("pass1", "pass2"))
    nb = n // 2 + 1
    roof = None
    L = s0["pass1_launches"]
    if L > 0:
        spl = s0["pass1_series"] / L
        pair_ms = (s0["pass1_ms"] + s0["pass2_ms"]) / L
        bps = nb * 8 / 2  # the template's bins, read once for both detectors of a segment
        alg = spl * bps
        # the fused launches run the kernels' multi-part instantiations: counters of their own only
        t1 = measured_traffic(f"{names[0]}_fused<{n1s},{n2s}>", spl)
        t2 = measured_traffic(f"{names[1]}_fused<{n1s},{n2s}>", spl)
        roof = {"bound": "hbm", "achieved": alg / (pair_ms * 1e-3) / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                "frac": alg / (pair_ms * 1e-3) / 1e9 / hbm_gbs,
                "traffic": (t1 + t2) if (t1 is not None and t2 is not None) else None,
                "kernel": f"fused filter {names[0]} + {names[1]} <{n1s},{n2s}> (all classes)",
                "per_launch_ms": pair_ms, "series_per_launch": spl, "bytes_per_series": bps,
                "launch_pairs_timed": L, "pass1_ms_per_launch": s0["pass1_ms"] / L,
                "pass2_ms_per_launch": s0["pass2_ms"] / L,
                "bytes_convention": "the template's one-sided FD bins, read once and shared by both detectors of a "
                                    "segment (4,096 B per template-second at 2048 Hz, FP32 bank); time = the two "
                                    "passes per launch pair (CUDA events around the fused launches)",
                "profile_stride": PROFILE_STRIDE,
                "peak_kind": f"{hbm_kind} HBM copy bandwidth"}
    series_step = sum(n_tmpl[ci] * seg[ci]["n_seg"] * 2 for ci in range(n_cls))
    step_bytes = series_step * nb * 8 / 2
    step_hbm = step_bytes / (t_dev / args.steps) / 1e9

    e2e = None
    if not args.no_e2e:  # public API from pinned host strain, triggers read back every step
        pinned = x.cpu().pin_memory()
        xd = torch.empty_like(x)
        te, d2h = [], 0
        for it in range(args.steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(st):
                xd.copy_(pinned, non_blocking=True)
            b.run(xd, mode=mode)
            trig, n_found, _ = b.triggers()
            if it > 0:  # the first pass warms this path up
                te.append(time.perf_counter() - t0)
                d2h += trig.nbytes
        e_val = td_step * args.steps / sum(te)
        if dist is not None:
            t_e, td_e_all = reduce_timing(dist, sum(te), td_step * args.steps, dev)
            e_val = td_e_all / t_e
        e2e = {"value": e_val, "unit": UNIT, "h2d_bytes_per_step": int(pinned.numel() * 4),
               "d2h_bytes_per_step": int(d2h / args.steps)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        xh = x.cpu().numpy().astype(np.float64)
        pool = OraclePool(c, init=_pool_init_uneven, work=_pool_work_uneven, initargs=(c, xh, n))
        try:
            rate, k, el = pool.run(args.cpu_seconds)
        finally:
            pool.close()
        cpu = {"value": rate, "unit": UNIT, "cores": pool.n, "kind": "oracle",
               "sample": f"oracle segmented_filter (numpy FP64) in {pool.n} processes, one per host core: {k} "
                         f"templates spread over the length classes, each over the whole 2 x 4096 s stream in "
                         f"segments of {n} samples, {el:.1f} s; CPU {cpu_model()}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "f16": "f32 + f16 (f16 intermediate and tensor-core operands)",
                      "f16x2": "f32 + f16 pairs (hi + lo intermediate and tensor-core operands)"}[args.intermediate],
            "data": "synthetic",
            "config": {"workload": WORKLOAD_UNEVEN, "intermediate": args.intermediate, "segment_n": n,
                       "segments_per_class": [g["n_seg"] for g in seg], "templates_per_class": n_tmpl,
                       "series_per_step": series_step, "td_seconds_per_step": td_step,
                       "l2": "512 MB buffer written between timed steps; banks (84 GB) streamed from HBM",
                       "run_mode": "MF_RUN_FUSED", "parallelism": f"{world} independent streams (one per GPU)"},
            "roofline": roof,
            "hbm_step": {"template_bytes_per_step": step_bytes, "achieved_gbs": step_hbm, "peak_gbs": hbm_gbs,
                         "frac": step_hbm / hbm_gbs, "peak_kind": hbm_kind},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(sum(s_["launches"] for s_ in sts)),
            "clocks": clk,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    b.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.kernel_case:
        return kernel_case(args.kernel_case, args.kernel_templates, args.intermediate)
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.workload == "uneven":
        return uneven_main(args, rank, world, local)

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
    if args.small:
        nb_ptr, nb_idx = cfg.nbhd_ptr, cfg.nbhd_idx
    else:  # set-up, untimed: neighbourhoods from the exact match >= 0.9, computed with the filter
        from paper_2309_00019_gb300.nbhd import exact_nbhd_of_config
        nb_ptr, nb_idx, _ = exact_nbhd_of_config(cfg.coarse_m1, cfg.coarse_m2, cfg.fine_m1, cfg.fine_m2, cfg.f_low,
                                                 cfg.fs2, device=dev)
    h = Hierarchy(hp, cfg.psd1, cfg.psd2, len(cfg.coarse_m1), len(cfg.fine_m1), nb_ptr, nb_idx, device=dev)
    if args.intermediate != "f32":
        h.p2.set_intermediate(mf.MF_F16 if args.intermediate == "f16" else mf.MF_F16X2)
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
        p.profile(PROFILE_STRIDE)
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

    # the fused filter (k_cols + k_rows launch pairs profiled in the timed region): HBM roofline of the
    # template bytes it must stream, and the ALU view of its dominant kernel
    hbm_gbs, hbm_kind = peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max_mhz = clk.get("sm_max_mhz") or 2070.0
    alu_derived = n_sm * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    try:  # measured FP32 FMA throughput: the ALU peak
        alu_probe = mf.fma_probe()
    except Exception:
        alu_probe = None
    alu_peak = alu_probe or alu_derived
    kinds, pairs = [], []
    for stage, s, n, plan in (("stage1", s1, hp.n1, h.p1), ("stage2", s2, hp.n2, h.p2)):
        lg = int(round(math.log2(n)))
        n1s, n2s = 1 << ((lg + 1) // 2), 1 << (lg // 2)
        names = KERNEL_NAMES.get(s["impl"], ("pass1", "pass2"))
        nb = n // 2 + 1
        eb = 8 if plan.desc.dtype == mf.MF_F32 else 4  # bytes per stored template bin
        for k, sub, nm in (("pass1", n1s, names[0]), ("pass2", n2s, names[1])):
            if s[f"{k}_launches"] > 0:
                kinds.append(dict(kernel=f"{nm}<{n1s},{n2s}> ({stage})", ms=s[f"{k}_ms"],
                                  launches=s[f"{k}_launches"], series=s[f"{k}_series"],
                                  flops_series=5.0 * n * math.log2(sub), n=n))
        L = s["pass1_launches"]
        if L > 0 and s["pass2_launches"] == L:
            spl = s["pass1_series"] / L
            pair_ms = (s["pass1_ms"] + s["pass2_ms"]) / L
            alg = spl * nb * eb / hp.n_det  # the template's bins, read once for all detectors
            t1 = measured_traffic(f"{names[0]}<{n1s},{n2s}>", spl)
            t2 = measured_traffic(f"{names[1]}<{n1s},{n2s}>", spl)
            pairs.append(dict(kernel=f"{names[0]} + {names[1]} <{n1s},{n2s}> ({stage})",
                              ms_total=s["pass1_ms"] + s["pass2_ms"], launch_pairs=L, series_per_launch=spl,
                              per_launch_pair_ms=pair_ms, algorithmic_bytes_per_pair=alg,
                              bytes_per_series=nb * eb / hp.n_det,
                              achieved_gbs=alg / (pair_ms * 1e-3) / 1e9,
                              traffic=(t1 + t2) if (t1 is not None and t2 is not None) else None))
    roof = roof_alu = None
    if pairs:
        dp = max(pairs, key=lambda d: d["ms_total"])
        roof = {"bound": "hbm", "achieved": dp["achieved_gbs"], "peak": hbm_gbs, "unit": "GB/s",
                "frac": dp["achieved_gbs"] / hbm_gbs, "traffic": dp["traffic"],
                "kernel": "fused filter " + dp["kernel"], "per_launch_ms": dp["per_launch_pair_ms"],
                "series_per_launch": dp["series_per_launch"], "bytes_per_series": dp["bytes_per_series"],
                "bytes_convention": "the template's one-sided FD bins, read once and shared by both detectors "
                                    "(FP32: 4,096 B per template-second at 2048 Hz); time = k_cols + k_rows per "
                                    "launch pair (CUDA events on the plan's stream, every profile_stride-th pair "
                                    "of the timed steps)",
                "peak_kind": f"{hbm_kind} HBM copy bandwidth", "profile_stride": PROFILE_STRIDE, "filters": pairs}
    if kinds:
        dom = max(kinds, key=lambda d: d["ms"])
        per_launch_ms = dom["ms"] / dom["launches"]
        spl = dom["series"] / dom["launches"]
        achieved = spl * dom["flops_series"] / (per_launch_ms * 1e-3) / 1e12
        klist = [{"kernel": d["kernel"], "launches": d["launches"], "ms_total": d["ms"],
                  "per_launch_ms": d["ms"] / d["launches"], "series_per_launch": d["series"] / d["launches"],
                  "alu_tflops": d["series"] / d["launches"] * d["flops_series"] / (d["ms"] / d["launches"] * 1e-3)
                  / 1e12} for d in kinds]
        roof_alu = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved / alu_peak, "kernel": dom["kernel"], "per_launch_ms": per_launch_ms,
                    "series_per_launch": spl, "flops_per_series": dom["flops_series"],
                    "flop_convention": "5 N log2(M) per series for an N-point transform built from M-point sub-FFTs",
                    "peak_kind": "measured FP32 FMA probe (mf_fma_probe)" if alu_probe else "derived",
                    "derived_peak": alu_derived,
                    "derived_note": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {sm_max_mhz:.0f} MHz",
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
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "f16": "f32 + f16 (f16 intermediate and tensor-core operands)",
                      "f16x2": "f32 + f16 pairs (hi + lo intermediate and tensor-core operands)"}[args.intermediate],
            "data": "synthetic",
            "config": {"workload": WORKLOAD if not args.small else "scaled-down 32 s hierarchy (check run)",
                       "stage2_intermediate": args.intermediate,
                       "union_templates": int(statistics.mean(unions)),
                       "td_seconds_per_step": td_total / args.steps,
                       "l2": "512 MB buffer written between timed steps; banks (1 GB + 84 GB) streamed from HBM",
                       "parallelism": f"{world} independent segments (one per GPU)"},
            "roofline": roof,
            "roofline_alu": roof_alu,
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
