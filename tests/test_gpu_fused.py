"""GPU checks of the one-launch filter (both four-step passes of the whole
selection in one persistent kernel, Sec. V.C's one inverse FFT per template
and segment with the intermediate kept in an L2-resident ring): its triggers
are bit-identical to those of the two-launch path, which runs the same
arithmetic, across ring wrap-around, selections shorter than the queue lag,
subsets, 16-bit storage and both supported lengths; a sample of templates is
also checked against the FP64 oracle."""

import numpy as np
import pytest

import synth
from tests.parity import compare_triggers, oracle_rho2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def mf(lib):
    from paper_2309_00019_gb300 import mf as m
    return m


def _setup(lg, n_tmpl, seed):
    n = 1 << lg
    fs = 2048.0 if lg == 20 else 1024.0
    rng = np.random.default_rng(seed)
    psd = synth.psd_bins(n, fs)
    m1, m2 = synth.sample_bank_uniform_masses(rng, n_tmpl, 2.0, 12.0)
    fd = np.stack([synth.coloured_noise_fd(rng, n, fs) for _ in range(2)])
    i = min(1, n_tmpl - 1)  # the injected template
    amp = 10.0 / synth.taylorf2_norm_continuum(m1[i], m2[i], 30.0, fs / 2)
    fd[1] += synth.taylorf2(n, fs, m1[i], m2[i], 30.0, t0=0.41 * n / fs, amp=amp)
    return n, fs, psd, m1, m2, fd.astype(np.complex64)


def _run(mf, n, fs, psd, bank_dev, dt, mode, batch=None, subset=None, dtype=0, data16=False):
    p = mf.Plan(fs, n, 2, 30.0, fs / 2, 3.2, int(fs) // 2, dtype=dtype, max_triggers=1 << 22)
    p.set_psd(psd)
    if batch is not None:
        p.set_batch(batch)
    p.set_filter_mode(mode)
    if dtype == 0:
        p.load_bank(bank_dev)
    else:
        p.bank_reserve(bank_dev.shape[0], dtype)
        p.bank_quantize_rows(0, bank_dev, ld=bank_dev.shape[1], on_device=1)
        if data16:
            p.set_data_dtype(dtype)
    p.profile(True)
    p.filter(dt, subset=None if subset is None else torch.from_numpy(subset).to(DEV))
    trig, cnt, _ = p.triggers()
    st = p.stats(reset=True)
    p.close()
    assert cnt == len(trig) > 0
    return trig, st


@pytest.mark.parametrize("lg,n_tmpl,batch", [(18, 23, None), (18, 5, 3), (20, 11, None), (20, 1, None),
                                             (20, 2, None), (20, 7, 3), (20, 9, 2)])
def test_fused_matches_two_launch_path_bitwise(mf, lg, n_tmpl, batch):
    n, fs, psd, m1, m2, fd = _setup(lg, n_tmpl, 300 + lg + n_tmpl)
    bank = synth.taylorf2_torch(n, fs, m1, m2, 30.0, DEV)
    dt = torch.from_numpy(fd).to(DEV)
    t2, s2 = _run(mf, n, fs, psd, bank, dt, mf.MF_FILTER_TWO_PASS, batch)
    t1, s1 = _run(mf, n, fs, psd, bank, dt, mf.MF_FILTER_FUSED, batch)
    assert s2["impl"] == 2 and s2["pass1_launches"] >= 1 and s2["fused_launches"] == 0
    assert s1["impl"] == 3 and s1["fused_launches"] == 1 and s1["pass1_launches"] == 0
    assert s1["fused_series"] == 2 * n_tmpl
    assert np.array_equal(t1, t2)
    print(f"\nN=2^{lg}, {n_tmpl} templates, batch {batch}: {len(t1)} identical triggers; "
          f"fused {s1['fused_ms']:.3f} ms, two-launch {s2['pass1_ms'] + s2['pass2_ms']:.3f} ms")


def test_fused_subset_16bit_and_fallback(mf):
    lg, n_tmpl = 18, 17
    n, fs, psd, m1, m2, fd = _setup(lg, n_tmpl, 77)
    bank = synth.taylorf2_torch(n, fs, m1, m2, 30.0, DEV)
    dt = torch.from_numpy(fd).to(DEV)
    sub = np.array([16, 0, 3, 4, 9, 1, 12, 8], dtype=np.int32)
    t2, _ = _run(mf, n, fs, psd, bank, dt, mf.MF_FILTER_TWO_PASS, subset=sub)
    t1, s1 = _run(mf, n, fs, psd, bank, dt, mf.MF_FILTER_FUSED, subset=sub)
    assert s1["impl"] == 3 and np.array_equal(t1, t2)
    assert set(np.unique(t1["tmpl"])) <= set(sub.tolist())
    for dtype in (1, 2):
        a, _ = _run(mf, n, fs, psd, bank, dt, mf.MF_FILTER_TWO_PASS, dtype=dtype, data16=True)
        b, sb = _run(mf, n, fs, psd, bank, dt, mf.MF_FILTER_FUSED, dtype=dtype, data16=True)
        assert sb["impl"] == 3 and np.array_equal(a, b)
    # a ring of one template leaves pass 1 nothing to run ahead into: the plan keeps two launches per batch
    t3, s3 = _run(mf, n, fs, psd, bank, dt, mf.MF_FILTER_FUSED, batch=1)
    assert s3["impl"] == 2 and s3["fused_launches"] == 0
    t4, _ = _run(mf, n, fs, psd, bank, dt, mf.MF_FILTER_TWO_PASS, batch=1)
    assert np.array_equal(t3, t4)
    # the smallest ring, two templates
    t5, s5 = _run(mf, n, fs, psd, bank, dt, mf.MF_FILTER_FUSED, batch=2)
    assert s5["impl"] == 3 and np.array_equal(t5, t4)


def test_fused_against_fp64_oracle_at_2e20(mf):
    """Nine templates (the ring of four wraps twice), two detectors: the
    templates 0, 1 (the injection) and 8 against the FP64 oracle."""
    lg, n_tmpl = 20, 9
    n, fs, psd, m1, m2, fd = _setup(lg, n_tmpl, 5)
    bank = synth.taylorf2_torch(n, fs, m1, m2, 30.0, DEV)
    trig, st = _run(mf, n, fs, psd, bank, torch.from_numpy(fd).to(DEV), mf.MF_FILTER_FUSED)
    assert st["impl"] == 3
    ids = [0, 1, 8]
    rows = bank[ids].cpu().numpy().astype(np.complex128)
    rho2, _ = oracle_rho2(fd.astype(np.complex128), rows, psd, n, fs, 30.0, fs / 2)
    sub = trig[np.isin(trig["tmpl"], ids)]
    s = compare_triggers(sub, rho2, ids, 3.2, int(fs) // 2)
    assert s["exact"] >= 0.99 * len(sub)
    inj = sub[(sub["tmpl"] == 1) & (sub["det"] == 1)]
    j0 = int(round(0.41 * n))
    assert np.abs(inj["sample"].astype(np.int64) - j0).min() <= 1
