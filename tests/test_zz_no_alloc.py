"""mf_filter_noalloc, the entry point for callers that cannot allocate GPU
memory (it keeps its working memory in a static device array), must give the
same triggers as the plan-based mf_filter on the same inputs, on two calls in
a row (the array keeps the previous call's contents, so each call has to
clear what must start at zero).  Collected last so that a failure here stops
a -x run only after every other test has run."""

import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _inputs(seed):
    n, fs, n_tmpl = 1 << 14, 512.0, 48
    rng = np.random.default_rng(seed)
    psd = synth.psd_bins(n, fs)
    m1, m2 = synth.sample_bank_uniform_masses(rng, n_tmpl, 1.4, 10.0)
    bank = np.stack([synth.taylorf2(n, fs, a, b, 30.0, dtype=np.complex64) for a, b in zip(m1, m2)])
    fd = np.stack([synth.coloured_noise_fd(rng, n, fs) for _ in range(2)])
    amp = 10.0 / synth.taylorf2_norm_continuum(m1[5], m2[5], 30.0, fs / 2)
    fd[1] += synth.taylorf2(n, fs, m1[5], m2[5], 30.0, t0=11.0, amp=amp)
    return n, fs, psd, bank, fd.astype(np.complex64)


def _keyed(trig):
    return {(int(t["det"]), int(t["tmpl"]), int(t["sample"])): float(t["snr"]) for t in trig}


def test_noalloc_matches_plan_filter_on_two_calls(lib):
    from paper_2309_00019_gb300 import mf

    thr, window = 4.0, 256
    for call, seed in enumerate((21, 22)):
        n, fs, psd, bank, fd = _inputs(seed)
        nb = n // 2 + 1
        plan = mf.Plan(fs, n, 2, 30.0, fs / 2, thr, window)
        plan.set_psd(psd)
        plan.load_bank(bank)
        d = torch.from_numpy(fd).to(DEV)
        plan.filter(d)
        ref, n_ref, _ = plan.triggers()
        plan.close()

        cap = 1 << 16
        out = torch.zeros(cap * 24, dtype=torch.uint8, device=DEV)
        count = torch.full((1,), -1, dtype=torch.int64, device=DEV)
        psd_d = torch.from_numpy(psd).to(DEV)
        bank_d = torch.from_numpy(bank).to(DEV)
        st = lib.mf_filter_noalloc(fs, n, 2, 30.0, fs / 2, thr, window, C.c_void_p(psd_d.data_ptr()),
                                   C.c_void_p(bank_d.data_ptr()), len(bank), nb, C.c_void_p(d.data_ptr()), nb,
                                   C.c_void_p(out.data_ptr()), cap, C.c_void_p(count.data_ptr()), None)
        assert st == mf.MF_OK, lib.mf_last_error(None)
        torch.cuda.synchronize()
        n_got = int(count.item())
        got = np.frombuffer(out.cpu().numpy().tobytes(), dtype=mf.TRIGGER_NP)[:n_got]
        assert n_got == n_ref > 0, (call, n_got, n_ref)
        a, b = _keyed(got), _keyed(ref)
        assert a.keys() == b.keys()
        for k in a:
            assert abs(a[k] - b[k]) <= 1e-4 * b[k]
        # ordered by (det, tmpl, sample) like mf_get_triggers
        keys = [(int(t["det"]), int(t["tmpl"]), int(t["sample"])) for t in got]
        assert keys == sorted(keys)


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
