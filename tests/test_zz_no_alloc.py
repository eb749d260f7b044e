"""mf_filter_noalloc, the entry point for callers that cannot allocate GPU
memory (it keeps its working memory in a static device array instead of
asking for any), checked against the FP64 oracle with the documented
near-tie allowances, and against the plan-based mf_filter on the same inputs
on two calls in a row (the array keeps the previous call's contents, so each
call has to clear what must start at zero).  Further cases cover the largest
layout of the array (N = 2^16, 1000 templates, so the templates go through
it in many batches), one detector with an analysis band below Nyquist, and a
trigger buffer smaller than the number found.  Collected last so that a
failure here stops a -x run only after every other test has run."""

import ctypes as C

import numpy as np
import pytest

import synth
from tests.parity import compare_triggers, oracle_rho2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
F_LOW = 30.0


def _inputs(seed, n, fs, n_tmpl, n_det, inj=5):
    rng = np.random.default_rng(seed)
    psd = synth.psd_bins(n, fs)
    m1, m2 = synth.sample_bank_uniform_masses(rng, n_tmpl, 1.4, 10.0)
    bank = synth.taylorf2_torch(n, fs, m1, m2, F_LOW, DEV).cpu().numpy()  # complex64 [n_tmpl][N/2+1]
    fd = np.stack([synth.coloured_noise_fd(rng, n, fs) for _ in range(n_det)])
    amp = 10.0 / synth.taylorf2_norm_continuum(m1[inj], m2[inj], F_LOW, fs / 2)
    fd[n_det - 1] += synth.taylorf2(n, fs, m1[inj], m2[inj], F_LOW, t0=0.35 * n / fs, amp=amp)
    return psd, bank, fd.astype(np.complex64)


def _noalloc(lib, fs, n, n_det, f_high, thr, window, psd, bank, fd, cap):
    from paper_2309_00019_gb300 import mf

    nb = n // 2 + 1
    out = torch.zeros(cap * mf.TRIGGER_NP.itemsize, dtype=torch.uint8, device=DEV)
    count = torch.full((1,), -1, dtype=torch.int64, device=DEV)
    psd_d = torch.from_numpy(psd).to(DEV)
    bank_d = torch.from_numpy(bank).to(DEV)
    d = torch.from_numpy(fd).to(DEV)
    st = lib.mf_filter_noalloc(fs, n, n_det, F_LOW, f_high, thr, window, C.c_void_p(psd_d.data_ptr()),
                               C.c_void_p(bank_d.data_ptr()), len(bank), nb, C.c_void_p(d.data_ptr()), nb,
                               C.c_void_p(out.data_ptr()), cap, C.c_void_p(count.data_ptr()), None)
    assert st == mf.MF_OK, lib.mf_last_error(None)
    torch.cuda.synchronize()
    n_found = int(count.item())
    got = np.frombuffer(out.cpu().numpy().tobytes(), dtype=mf.TRIGGER_NP)[:min(n_found, cap)].copy()
    return got, n_found


def _against_oracle(got, fd, bank, psd, n, fs, f_high, thr, window, chunk=64):
    """compare_triggers over every template, a chunk of oracle series at a time."""
    tot = dict(exact=0, tie_swaps=0, edge=0, max_rel_snr=0.0)
    for t0 in range(0, len(bank), chunk):
        ids = list(range(t0, min(t0 + chunk, len(bank))))
        rho2, _ = oracle_rho2(fd.astype(np.complex128), bank[ids].astype(np.complex128), psd, n, fs, F_LOW, f_high)
        st = compare_triggers(got[np.isin(got["tmpl"], ids)], rho2, ids, thr, window)
        for k in ("exact", "tie_swaps", "edge"):
            tot[k] += st[k]
        tot["max_rel_snr"] = max(tot["max_rel_snr"], st["max_rel_snr"])
    return tot


def _keys(trig):
    return [(int(t["det"]), int(t["tmpl"]), int(t["sample"])) for t in trig]


def test_noalloc_matches_oracle_and_mf_filter_on_two_calls(lib):
    from paper_2309_00019_gb300 import mf

    n, fs, thr, window = 1 << 14, 512.0, 4.0, 256
    for call, seed in enumerate((21, 22)):
        psd, bank, fd = _inputs(seed, n, fs, 48, 2)
        got, n_got = _noalloc(lib, fs, n, 2, fs / 2, thr, window, psd, bank, fd, 1 << 16)
        assert n_got == len(got) > 0
        assert _keys(got) == sorted(_keys(got))  # ordered by (det, tmpl, sample) like mf_get_triggers
        st = _against_oracle(got, fd, bank, psd, n, fs, fs / 2, thr, window)
        assert st["exact"] > 0

        plan = mf.Plan(fs, n, 2, F_LOW, fs / 2, thr, window)
        plan.set_psd(psd)
        plan.load_bank(bank)
        plan.filter(torch.from_numpy(fd).to(DEV))
        ref, n_ref, _ = plan.triggers()
        plan.close()
        # the two entry points agree to the tests' SNR tolerance on every common window peak; a window
        # present in one set only is an oracle near-tie at the threshold (both sets passed compare_triggers)
        a = {k: float(t["snr"]) for k, t in zip(_keys(got), got)}
        b = {k: float(t["snr"]) for k, t in zip(_keys(ref), ref)}
        common = a.keys() & b.keys()
        assert len(common) >= 0.99 * max(len(a), len(b)), (call, len(a), len(b), len(common))
        for k in common:
            assert abs(a[k] - b[k]) <= 2e-4 * b[k], (call, k, a[k], b[k])
        print(f"\ncall {call}: {n_got} triggers, oracle {st}, {len(common)} in common with mf_filter")


def test_noalloc_largest_layout_many_batches(lib):
    # N = 2^16, 2 detectors, 1000 templates and 32 windows: the weights, data, window maxima and
    # per-batch transform scratch fill the array, and the bank goes through it about 30 templates at a time
    n, fs, thr, window = 1 << 16, 2048.0, 4.5, 2048
    psd, bank, fd = _inputs(31, n, fs, 1000, 2, inj=777)
    got, n_got = _noalloc(lib, fs, n, 2, fs / 2, thr, window, psd, bank, fd, 1 << 18)
    assert n_got == len(got) > 0
    # templates of every batch (about 30 templates each) fired
    fired = np.zeros(1000, dtype=bool)
    fired[got["tmpl"]] = True
    assert fired.sum() > 800 and all(fired[b:b + 25].any() for b in range(0, 1000, 25))
    st = _against_oracle(got, fd, bank, psd, n, fs, fs / 2, thr, window)
    assert st["exact"] > 0
    print(f"\nN = 2^16, 1000 templates: {n_got} triggers, oracle {st}")


def test_noalloc_one_detector_band_below_nyquist_and_small_buffer(lib):
    n, fs, thr, window, f_high = 1 << 13, 512.0, 3.5, 128, 200.0
    psd, bank, fd = _inputs(41, n, fs, 40, 1)
    full, n_full = _noalloc(lib, fs, n, 1, f_high, thr, window, psd, bank, fd, 1 << 15)
    assert n_full == len(full) > 200
    st = _against_oracle(full, fd, bank, psd, n, fs, f_high, thr, window)
    assert st["exact"] > 0
    # a buffer smaller than the number found: count is still the full number, and the buffer holds the
    # first trig_cap triggers of the ordered list
    cap = 100
    part, n_part = _noalloc(lib, fs, n, 1, f_high, thr, window, psd, bank, fd, cap)
    assert n_part == n_full and len(part) == cap
    assert _keys(part) == _keys(full)[:cap]
    assert np.array_equal(part["snr"], full["snr"][:cap])
    print(f"\n1 detector, f_high {f_high} Hz: {n_full} triggers, oracle {st}")


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    from paper_2309_00019_gb300 import mf

    dummy = torch.zeros(16, device=DEV)
    p = C.c_void_p(dummy.data_ptr())
    # N above the 2^16 limit
    assert lib.mf_filter_noalloc(2048.0, 1 << 18, 1, 30.0, 1024.0, 5.0, 2048, p, p, 1, (1 << 17) + 1, p,
                                 (1 << 17) + 1, p, 1, p, None) == mf.MF_EINVAL
    assert b"2^16" in lib.mf_last_error(None)
    # too many templates
    assert lib.mf_filter_noalloc(512.0, 1 << 12, 1, 30.0, 256.0, 5.0, 512, p, p, 5000, 2049, p, 2049, p, 1, p,
                                 None) == mf.MF_EINVAL
    # too many windows per segment
    assert lib.mf_filter_noalloc(512.0, 1 << 14, 1, 30.0, 256.0, 5.0, 32, p, p, 1, 8193, p, 8193, p, 1, p,
                                 None) == mf.MF_EINVAL
