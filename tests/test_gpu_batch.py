"""GPU checks of the length-class runner (long data in overlapping segments,
Sec. V.C): triggers against the oracle's segmented search, the run modes
(serial, concurrent streams, captured CUDA graph, and the fused work queue over
all classes with its graph) against each other, the autotuners' choices, and
the full uneven-length workload (20,000 templates in 4/16/64/256 s classes over
2 x 4096 s at 2048 Hz) in every mode, FP32 and with the FP16 intermediate, with
sampled oracle checks."""

import math
import time

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def mf(lib):
    from paper_2309_00019_gb300 import mf as m
    return m


def compare_lists(gpu, ref, thr, window, snr_rtol=1e-4):
    """GPU vs oracle trigger lists of one class: the same (det, tmpl, window)
    set apart from windows whose peak is within snr_rtol of the threshold; in
    shared windows the peak SNR agrees to snr_rtol and the sample is the same
    unless another sample of the window is within snr_rtol of the peak (then
    the two SNRs still agree)."""
    def keyed(t):
        return {(int(x["det"]), int(x["tmpl"]), int(x["sample"]) // window): x for x in t}
    g, r = keyed(gpu), keyed(ref)
    assert len(g) == len(gpu) and len(r) == len(ref)
    for k in set(g) ^ set(r):
        x = g.get(k, r.get(k))
        assert abs(float(x["snr"]) - thr) <= snr_rtol * thr, (k, x)
    worst, moved = 0.0, 0
    for k in set(g) & set(r):
        rel = abs(float(g[k]["snr"]) - float(r[k]["snr"])) / float(r[k]["snr"])
        worst = max(worst, rel)
        moved += int(g[k]["sample"] != r[k]["sample"])
    assert worst <= snr_rtol, worst
    return dict(common=len(set(g) & set(r)), only=len(set(g) ^ set(r)), max_rel=worst, moved=moved)


def _small():
    return synth.make_config3(seed=5, n_tmpl=24, T=256.0, fs=512.0, f_low=40.0, class_len=(2.0, 8.0, 32.0), n_inj=6)


def _batch(mf, c, stream=None):
    b = mf.Batch(c.fs, 2, c.n_samples, c.f_low, c.fs / 2, c.thr, c.window, c.class_len, stream=stream)
    b.set_psd(c.psd(c.n_fd), c.n_fd)
    return b


def _load_banks(b, c, numpy_rows=True):
    for ci in range(len(c.class_len)):
        ids = c.class_ids(ci)
        if len(ids) == 0:
            continue
        g = b.segment(ci)
        p = b.plan(ci)
        p.bank_reserve(len(ids))
        rows = synth.taylorf2_torch(g["n"], c.fs, c.m1[ids], c.m2[ids], c.f_low, DEV)
        p.bank_set_rows(0, rows, ld=rows.shape[1], on_device=1)


def test_small_batch_matches_oracle_segmented_search(mf):
    c = _small()
    x = c.strain(DEV)
    xh = x.cpu().numpy().astype(np.float64)
    b = _batch(mf, c)
    for ci, n in enumerate((4096, 8192, 32768)):
        b.set_segment(ci, n)
    _load_banks(b, c)
    b.run(x, mode=mf.MF_RUN_SERIAL)
    trig, n_found, _ = b.triggers()
    assert n_found == len(trig) > 0
    for ci in range(3):
        ids = c.class_ids(ci)
        g = b.segment(ci)
        assert g["tmpl_len"] == int(math.ceil(c.class_len[ci] * c.fs / c.window)) * c.window
        bank = synth.taylorf2_torch(g["n"], c.fs, c.m1[ids], c.m2[ids], c.f_low, DEV).cpu().numpy()
        ref = O.segmented_filter(xh, c.fs, synth.psd_bins(g["n"], c.fs), c.f_low, c.fs / 2,
                                 bank.astype(np.complex128), g["n"], int(c.class_len[ci] * c.fs), c.thr, c.window)
        got = trig[trig["cls"] == ci]
        st = compare_lists(got, ref, c.thr, c.window)
        assert st["common"] > 0
        print(f"\nclass {ci}: N={g['n']} segments={g['n_seg']} oracle {len(ref)} / gpu {len(got)} triggers, {st}")
    # the loudest trigger is an injection (the 24-template bank matches some of them only partly)
    loud = trig[np.argmax(trig["snr"])]
    assert np.abs(loud["sample"] / c.fs - c.inj["tc"]).min() < 0.1


def test_run_modes_agree_bitwise_and_graph_replays(mf):
    c = _small()
    x = c.strain(DEV)
    st = torch.cuda.Stream()
    b = _batch(mf, c, stream=st.cuda_stream)
    for ci, n in enumerate((8192, 16384, 65536)):
        b.set_segment(ci, n)
    _load_banks(b, c)
    out = {}
    for mode in (mf.MF_RUN_SERIAL, mf.MF_RUN_STREAMS, mf.MF_RUN_GRAPH, mf.MF_RUN_GRAPH):
        b.run(x, mode=mode)
        out.setdefault(mode, []).append(b.triggers()[0])
    ref = out[mf.MF_RUN_SERIAL][0]
    assert len(ref) > 0
    for mode, lst in out.items():
        for t in lst:
            assert np.array_equal(t, ref), mode
    # another strain buffer: the graph is captured again for it
    x2 = x.clone()
    b.run(x2, mode=mf.MF_RUN_GRAPH)
    assert np.array_equal(b.triggers()[0], ref)


def test_autotune_picks_admissible_segments(mf):
    c = _small()
    x = c.strain(DEV)
    b = _batch(mf, c)
    n_tmpl = [len(c.class_ids(i)) for i in range(3)]
    b.autotune(n_tmpl)
    for ci in range(3):
        g = b.segment(ci)
        assert g["n"] >= 4096 and g["n"] & (g["n"] - 1) == 0
        assert g["stride"] > 0 and g["tmpl_len"] + g["stride"] <= g["n"] and g["stride"] % c.window == 0
        assert g["est_ms"] > 0
    _load_banks(b, c)
    b.run(x, mode=mf.MF_RUN_GRAPH)
    trig = b.triggers()[0]
    xh = x.cpu().numpy().astype(np.float64)
    for ci in range(3):
        ids = c.class_ids(ci)
        g = b.segment(ci)
        bank = synth.taylorf2_torch(g["n"], c.fs, c.m1[ids], c.m2[ids], c.f_low, DEV).cpu().numpy()
        ref = O.segmented_filter(xh, c.fs, synth.psd_bins(g["n"], c.fs), c.f_low, c.fs / 2,
                                 bank.astype(np.complex128), g["n"], int(c.class_len[ci] * c.fs), c.thr, c.window)
        compare_lists(trig[trig["cls"] == ci], ref, c.thr, c.window)


def test_autotune_fused_picks_one_length_and_runs_fused(mf):
    """The common-N autotuner gives every class with templates the same admissible segment length; at it the
    fused graph and the serial per-class run agree bit for bit."""
    c = _small()
    x = c.strain(DEV)
    st = torch.cuda.Stream()
    b = _batch(mf, c, stream=st.cuda_stream)
    n_tmpl = [len(c.class_ids(i)) for i in range(3)]
    b.autotune(n_tmpl, fused=True)
    seg = [b.segment(ci) for ci in range(3)]
    assert len({g["n"] for g, k in zip(seg, n_tmpl) if k > 0}) == 1
    for g in seg:
        assert g["stride"] > 0 and g["tmpl_len"] + g["stride"] <= g["n"] and g["est_ms"] > 0
    _load_banks(b, c)
    b.run(x, mode=mf.MF_RUN_SERIAL)
    ref = b.triggers()[0]
    b.run(x)  # default: the fused graph, since the classes share N
    assert np.array_equal(b.triggers()[0], ref) and len(ref) > 0


def test_config3_uneven_lengths_full_size(mf):
    """20,000 templates, 2 x 4096 s at 2048 Hz: autotuned segment lengths, the
    three run modes timed, and 2 templates per class checked by the oracle's
    segmented search."""
    c = synth.make_config3()
    x = c.strain(DEV)
    st = torch.cuda.Stream()
    b = _batch(mf, c, stream=st.cuda_stream)
    n_cls = len(c.class_len)
    b.autotune([len(c.class_ids(i)) for i in range(n_cls)])
    for ci in range(n_cls):
        ids = c.class_ids(ci)
        g = b.segment(ci)
        p = b.plan(ci)
        p.bank_reserve(len(ids))
        ld = (g["n"] // 2 + 1 + 63) // 64 * 64
        for r0, rows in synth.taylorf2_chunks_torch(g["n"], c.fs, c.m1[ids], c.m2[ids], c.f_low, DEV, chunk=256,
                                                    ld=ld):
            p.bank_set_rows(r0, rows, ld=ld, on_device=1)
    times = {}
    res = {}
    for name, mode in (("serial", mf.MF_RUN_SERIAL), ("streams", mf.MF_RUN_STREAMS), ("graph", mf.MF_RUN_GRAPH)):
        b.run(x, mode=mode)  # warm-up (and capture)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(3):
            b.run(x, mode=mode)
        e1.record(st)
        e1.synchronize()
        times[name] = e0.elapsed_time(e1) / 3
        res[name] = b.triggers()[0]
    for name in ("streams", "graph"):
        assert np.array_equal(res[name], res["serial"]), name
    trig = res["serial"]
    td = sum(len(c.class_ids(i)) for i in range(n_cls)) * 2 * (c.n_samples / c.fs)
    print("\nconfig 3: " + ", ".join(f"{k} {v:.1f} ms ({td / v * 1e3:.3g} template-s/s)" for k, v in times.items()))
    for ci in range(n_cls):
        g = b.segment(ci)
        print(f"  class {c.class_len[ci]:g} s: {len(c.class_ids(ci))} templates, N = {g['n']}, "
              f"{g['n_seg']} segments, stride {g['stride'] / c.fs:g} s, est {g['est_ms']:.1f} ms, serial run "
              f"{g['run_ms']:.1f} ms")
    # oracle on a sample: the 2 templates of each class with the most triggers
    xh = x.cpu().numpy().astype(np.float64)
    for ci in range(n_cls):
        ids = c.class_ids(ci)
        tc = trig[trig["cls"] == ci]
        cnt = np.bincount(tc["tmpl"], minlength=len(ids))
        pick = np.argsort(-cnt, kind="stable")[:2]
        g = b.segment(ci)
        bank = synth.taylorf2_torch(g["n"], c.fs, c.m1[ids[pick]], c.m2[ids[pick]], c.f_low, DEV).cpu().numpy()
        ref = O.segmented_filter(xh, c.fs, synth.psd_bins(g["n"], c.fs), c.f_low, c.fs / 2,
                                 bank.astype(np.complex128), g["n"], int(c.class_len[ci] * c.fs), c.thr, c.window)
        ref["tmpl"] = pick[ref["tmpl"]]
        got = tc[np.isin(tc["tmpl"], pick)]
        s = compare_lists(got, ref, c.thr, c.window)
        print(f"  class {ci} oracle sample (templates {list(pick)}): {s}")


def _launches(plans):
    return [p.stats(reset=True)["launches"] for p in plans]


def test_fused_work_queue_matches_per_class_bitwise(mf):
    """MF_RUN_FUSED: one launch pair per S series of the (class, template,
    segment, detector) queue, across class boundaries; its triggers and those
    of its captured graph are the per-class runs', bit for bit."""
    c = _small()
    x = c.strain(DEV)
    st = torch.cuda.Stream()
    b = _batch(mf, c, stream=st.cuda_stream)
    per = (3, 2, 5)
    for ci in range(3):
        b.set_segment(ci, 32768, per[ci])
    _load_banks(b, c)
    plans = [b.plan(ci) for ci in range(3)]
    b.run(x, mode=mf.MF_RUN_SERIAL)
    ref = b.triggers()[0]
    assert len(ref) > 0 and len(np.unique(ref["cls"])) == 3
    rows = [b.segment(ci)["n_seg"] * 2 for ci in range(3)]
    S = max(p * r for p, r in zip(per, rows))
    n_series = sum(len(c.class_ids(ci)) * rows[ci] for ci in range(3))
    assert n_series > 2 * S  # several launch pairs, some across class boundaries
    _launches(plans)
    b.run(x, mode=mf.MF_RUN_STREAMS)
    assert np.array_equal(b.triggers()[0], ref)
    per_class = _launches(plans)
    for mode in (mf.MF_RUN_FUSED, mf.MF_RUN_FUSED_GRAPH, mf.MF_RUN_FUSED_GRAPH):
        b.run(x, mode=mode)
        assert np.array_equal(b.triggers()[0], ref), mode
    _launches(plans)
    b.run(x, mode=mf.MF_RUN_FUSED)
    assert np.array_equal(b.triggers()[0], ref)
    fused = _launches(plans)
    # an uncaptured fused pass counts every filter launch on the first class's plan; the other classes
    # launched only their spectra
    assert fused[0] >= 2 * math.ceil(n_series / S)
    assert all(fused[ci] < per_class[ci] for ci in (1, 2)), (fused, per_class)
    print(f"\nfused: {n_series} series, S = {S}, launches per plan {fused} (per class {per_class})")
    # a class at another segment length: a fused run is refused
    b.set_segment(0, 16384, 3)
    ids = c.class_ids(0)
    p0 = b.plan(0)
    p0.bank_reserve(len(ids))
    p0.bank_set_rows(0, synth.taylorf2_torch(16384, c.fs, c.m1[ids], c.m2[ids], c.f_low, DEV), ld=16384 // 2 + 1,
                     on_device=1)
    with pytest.raises(mf.MFError) as ei:
        b.run(x, mode=mf.MF_RUN_FUSED)
    assert ei.value.status == mf.MF_ESTATE


def test_fused_fp16_intermediate_matches_per_class(mf):
    """Every class at N = 2^20 with the FP16 intermediate and the tensor-core
    row pass: fused and per-class triggers agree bit for bit, and with the FP32
    fused run within the FP16 path's tolerance.  The data (3072 s at 512 Hz)
    fill the 2048 s segments, so that the noise matches the PSD the SNR is
    normalised by."""
    c = synth.make_config3(seed=5, n_tmpl=24, T=3072.0, fs=512.0, f_low=40.0, class_len=(2.0, 8.0, 32.0), n_inj=12)
    x = c.strain(DEV)
    st = torch.cuda.Stream()
    b = mf.Batch(c.fs, 2, c.n_samples, c.f_low, c.fs / 2, c.thr, c.window, c.class_len, stream=st.cuda_stream)
    b.set_psd(c.psd(1 << 20), 1 << 20)
    for ci, per in enumerate((2, 3, 1)):
        b.set_segment(ci, 1 << 20, per)
    _load_banks(b, c)
    assert all(b.segment(ci)["n_seg"] == 2 for ci in range(3))
    # rows written by torch just before the upload are complete when the class plan reads them
    for ci in range(3):
        assert np.all(b.plan(ci).sigmasq(len(c.class_ids(ci))) > 0), ci
    b.run(x, mode=mf.MF_RUN_FUSED)
    ref32 = b.triggers()[0]
    assert len(ref32) > 20 and len(np.unique(ref32["cls"])) >= 2
    for ci in range(3):
        b.plan(ci).set_intermediate(mf.MF_F16)
    b.run(x, mode=mf.MF_RUN_STREAMS)
    ref16 = b.triggers()[0]
    for mode in (mf.MF_RUN_FUSED, mf.MF_RUN_FUSED_GRAPH, mf.MF_RUN_FUSED_GRAPH):
        b.run(x, mode=mode)
        assert np.array_equal(b.triggers()[0], ref16), mode
    s = _compare_f16(ref16, ref32, c.thr, c.window)
    print(f"\nFP16 vs FP32 fused: {s}")
    # FP16 pairs with split products: fused and per class bit for bit, at the FP32 bar against FP32
    for ci in range(3):
        b.plan(ci).set_intermediate(mf.MF_F16X2)
    b.run(x, mode=mf.MF_RUN_STREAMS)
    ref2 = b.triggers()[0]
    for mode in (mf.MF_RUN_FUSED, mf.MF_RUN_FUSED_GRAPH):
        b.run(x, mode=mode)
        assert np.array_equal(b.triggers()[0], ref2), mode
    s = _compare_f16(ref2, ref32, c.thr, c.window, rel_tie=2e-4, snr_rtol=1e-4)
    print(f"FP16 pairs vs FP32 fused: {s}")


def _compare_f16(t16, t32, thr, window, rel_tie=2e-3, snr_rtol=1e-3):
    """FP16-intermediate triggers against FP32 ones: the same (class, det,
    template, window) set apart from windows within rel_tie of the threshold,
    SNR within snr_rtol in shared windows, at least 99% of the windows shared."""
    def keyed(t):
        return {(int(x["cls"]), int(x["det"]), int(x["tmpl"]), int(x["sample"]) // window): float(x["snr"]) for x in t}
    a, r = keyed(t16), keyed(t32)
    for k in set(a) ^ set(r):
        v = a.get(k, r.get(k))
        assert abs(v - thr) <= rel_tie * thr, (k, v)
    common = set(a) & set(r)
    worst = max((abs(a[k] - r[k]) / r[k] for k in common), default=0.0)
    assert worst <= snr_rtol, worst
    assert len(common) >= 0.99 * max(len(a), len(r))
    return dict(common=len(common), only=len(set(a) ^ set(r)), max_rel=worst)


def test_config3_fused_full_size(mf):
    """Config 3 (20,000 templates in 4/16/64/256 s classes, 2 x 4096 s at
    2048 Hz) with one segment length for every class (mf_batch_autotune_fused):
    the per-class modes, the fused work queue and its graph give identical
    triggers, timed; then the FP16 intermediate (tensor-core row pass), per class
    and fused, against FP32; one template per class checked by the oracle's
    segmented search."""
    c = synth.make_config3()
    x = c.strain(DEV)
    st = torch.cuda.Stream()
    b = _batch(mf, c, stream=st.cuda_stream)
    n_cls = len(c.class_len)
    b.autotune([len(c.class_ids(i)) for i in range(n_cls)], fused=True)
    seg = [b.segment(ci) for ci in range(n_cls)]
    assert len({g["n"] for g in seg}) == 1
    lib = mf.load()
    for ci in range(n_cls):
        ids = c.class_ids(ci)
        p = b.plan(ci)
        p.bank_reserve(len(ids))
        p.bank_generate_taylorf2(0, c.m1[ids], c.m2[ids], c.f_low)
    td = sum(len(c.class_ids(i)) for i in range(n_cls)) * 2 * (c.n_samples / c.fs)

    def timed(mode):
        b.run(x, mode=mode)  # warm-up (and capture)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(3):
            b.run(x, mode=mode)
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / 3, b.triggers()[0]

    times, res = {}, {}
    for name, mode in (("serial", mf.MF_RUN_SERIAL), ("streams", mf.MF_RUN_STREAMS), ("graph", mf.MF_RUN_GRAPH),
                       ("fused", mf.MF_RUN_FUSED), ("fused graph", mf.MF_RUN_FUSED_GRAPH)):
        times[name], res[name] = timed(mode)
        assert np.array_equal(res[name], res["serial"]), name
    for ci in range(n_cls):
        b.plan(ci).set_intermediate(mf.MF_F16)
    for name, mode in (("streams f16", mf.MF_RUN_STREAMS), ("fused f16", mf.MF_RUN_FUSED),
                       ("fused graph f16", mf.MF_RUN_FUSED_GRAPH)):
        times[name], res[name] = timed(mode)
        assert np.array_equal(res[name], res["streams f16"]), name
    s = _compare_f16(res["fused f16"], res["serial"], c.thr, c.window)
    print(f"\nconfig 3, N = {seg[0]['n']} for every class (segments {[g['n_seg'] for g in seg]}):")
    for k, v in times.items():
        print(f"  {k}: {v:.1f} ms ({td / v * 1e3:.3g} template-s/s)")
    print(f"  FP16 vs FP32: {s}")
    # oracle on a sample: the template of each class with the most triggers, its rows from the library's generator
    xh = x.cpu().numpy().astype(np.float64)
    n = seg[0]["n"]
    nb = n // 2 + 1
    for ci in range(n_cls):
        ids = c.class_ids(ci)
        for name, tol in (("serial", 1e-4), ("fused f16", 1e-3)):
            tc = res[name][res[name]["cls"] == ci]
            t = int(np.argmax(np.bincount(tc["tmpl"], minlength=len(ids))))
            row = torch.zeros((1, nb), dtype=torch.complex64, device=DEV)
            a1, a2 = np.array([c.m1[ids[t]]]), np.array([c.m2[ids[t]]])
            rc = lib.mf_taylorf2(a1.ctypes.data, a2.ctypes.data, 1, c.fs, n, c.f_low, mf._ptr(row), nb,
                                 torch.cuda.current_stream().cuda_stream)
            assert rc == mf.MF_OK
            torch.cuda.synchronize()
            bank = row.cpu().numpy().astype(np.complex128)
            ref = O.segmented_filter(xh, c.fs, synth.psd_bins(n, c.fs), c.f_low, c.fs / 2, bank, n,
                                     int(c.class_len[ci] * c.fs), c.thr, c.window)
            ref["tmpl"] = t
            st_ = compare_lists(tc[tc["tmpl"] == t], ref, c.thr, c.window, snr_rtol=tol)
            assert st_["common"] > 0
            print(f"  class {ci} {name} oracle sample (template {t}): {st_}")
