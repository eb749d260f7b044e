"""GPU parity of the CUDA matched filter (through the C ABI) against the FP64
oracle: spectra, template norms, trigger sets and SNRs on seeded synthetic
inputs at every supported FFT length, ragged windows and valid ranges,
noiseless injections and the edge cases of the selection."""

import math

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O
from tests.parity import compare_triggers, oracle_rho2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _plan(mf, fs, n, n_det, f_low, thr, window, f_high=None, vb=0, ve=None, max_trig=1 << 20, dtype=0):
    return mf.Plan(fs, n, n_det, f_low, fs / 2 if f_high is None else f_high, thr, window, vb, ve,
                   dtype=dtype, max_triggers=max_trig)


@pytest.fixture(scope="module")
def mf(lib):
    from paper_2309_00019_gb300 import mf as m
    return m


@pytest.mark.parametrize("lg", list(range(12, 21)))
def test_strain_to_fd_matches_fp64_rfft(mf, lg):
    n = 1 << lg
    fs = 512.0
    rng = np.random.default_rng(lg)
    x = rng.standard_normal((2, n)).astype(np.float32) * 1e-20
    p = _plan(mf, fs, n, 2, 20.0, 5.0, 512)
    out = torch.zeros((2, n // 2 + 1), dtype=torch.complex64, device=DEV)
    p.strain_to_fd(torch.from_numpy(x).to(DEV), out)
    got = out.cpu().numpy()
    ref = O.strain_to_fd(x, fs)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 2e-6 * math.sqrt(lg), err


def test_sigmasq_is_fp64_sum(mf):
    c = synth.make_config1()
    bank = c.bank()
    p = _plan(mf, c.fs, c.n, 1, c.f_low, c.thr, c.window)
    p.set_psd(c.psd)
    p.load_bank(torch.from_numpy(bank).to(DEV))
    w = O.weights(c.n, c.fs, c.f_low, c.f_high, c.psd)
    ref = O.sigmasq(bank.astype(np.complex128), w)
    assert np.allclose(p.sigmasq(), ref, rtol=1e-12, atol=0)
    # host-pointer bank load gives the same
    p2 = _plan(mf, c.fs, c.n, 1, c.f_low, c.thr, c.window)
    p2.set_psd(c.psd)
    p2.load_bank(bank)
    assert np.array_equal(p2.sigmasq(), p.sigmasq())


def test_config1_trigger_parity(mf):
    """One detector, 32 s @ 512 Hz, 64 TaylorF2 templates, injection SNR 12, thr 5.5, 1 s windows."""
    c = synth.make_config1()
    bank = c.bank()
    p = _plan(mf, c.fs, c.n, 1, c.f_low, c.thr, c.window)
    p.set_psd(c.psd)
    p.load_bank(torch.from_numpy(bank).to(DEV))
    dt = torch.zeros((1, c.n // 2 + 1), dtype=torch.complex64, device=DEV)
    p.strain_to_fd(torch.from_numpy(c.strain).to(DEV), dt)
    p.filter(dt)
    trig, n, st = p.triggers()
    assert st == mf.MF_OK and n == len(trig) > 0
    s = O.strain_to_fd(c.strain, c.fs)
    rho2, z = oracle_rho2(s, bank, c.psd, c.n, c.fs, c.f_low, c.f_high)
    stats = compare_triggers(trig, rho2, range(64), c.thr, c.window, snr_rtol=1e-4, phase_atol=4e-3, z=z)
    assert stats["exact"] == len(trig)
    # the injection is found where it was put, at SNR ~ 12 (the noise adds a little)
    k = (trig["tmpl"] == c.inj_tmpl) & (trig["sample"] == c.inj_sample)
    assert k.sum() == 1 and abs(trig["snr"][k][0] - 12.0) < 1.0
    # ordering (det, tmpl, sample)
    key = trig["det"].astype(np.int64) * 2**40 + trig["tmpl"].astype(np.int64) * 2**24 + trig["sample"]
    assert np.all(np.diff(key) > 0)


@pytest.mark.parametrize("lg", list(range(12, 21)))
def test_filter_parity_every_length(mf, lg):
    """Two detectors, low threshold (almost every window has a peak), TaylorF2 bank with an injection."""
    n = 1 << lg
    fs = 2048.0 if lg >= 17 else 512.0
    n_tmpl = 3 if lg >= 19 else 6
    rng = np.random.default_rng(100 + lg)
    psd = synth.psd_bins(n, fs)
    m1, m2 = synth.sample_bank_uniform_masses(rng, n_tmpl, 2.0, 12.0)
    bank = np.stack([synth.taylorf2(n, fs, a, b, 30.0, dtype=np.complex64) for a, b in zip(m1, m2)])
    fd = np.stack([synth.coloured_noise_fd(rng, n, fs) for _ in range(2)])
    amp = 9.0 / synth.taylorf2_norm_continuum(m1[1], m2[1], 30.0, fs / 2)
    fd[0] += synth.taylorf2(n, fs, m1[1], m2[1], 30.0, t0=0.37 * n / fs, amp=amp)
    strain = np.stack([synth.strain_from_fd(fd[d], n, fs) for d in range(2)]).astype(np.float32)
    W = int(fs) // 2
    p = _plan(mf, fs, n, 2, 30.0, 3.0, W)
    p.set_psd(psd)
    p.load_bank(torch.from_numpy(bank).to(DEV))
    dt = torch.zeros((2, n // 2 + 1), dtype=torch.complex64, device=DEV)
    p.strain_to_fd(torch.from_numpy(strain).to(DEV), dt)
    p.filter(dt)
    trig, ntrig, _ = p.triggers()
    s = O.strain_to_fd(strain, fs)
    rho2, _ = oracle_rho2(s, bank, psd, n, fs, 30.0, fs / 2)
    stats = compare_triggers(trig, rho2, range(n_tmpl), 3.0, W)
    assert stats["exact"] >= 0.99 * ntrig
    assert ntrig > 0.5 * 2 * n_tmpl * (n // W)


def test_noiseless_injection_recovers_optimal_snr(mf):
    n, fs = 1 << 16, 2048.0
    psd = synth.psd_bins(n, fs)
    h = synth.taylorf2(n, fs, 1.6, 1.3, 30.0)
    bank = h[None, :].astype(np.complex64)
    w = O.weights(n, fs, 30.0, fs / 2, psd)
    sig = math.sqrt(O.sigmasq(bank[0].astype(np.complex128), w))
    j0 = 12345
    k = np.arange(n // 2 + 1)
    A = 15.0 / sig
    s = (A * bank[0].astype(np.complex128) * np.exp(-2j * math.pi * k * j0 / n) * np.exp(0.3j))
    p = _plan(mf, fs, n, 1, 30.0, 5.0, 2048)
    p.set_psd(psd)
    p.load_bank(bank)
    p.filter(torch.from_numpy(s.astype(np.complex64)[None]).to(DEV))
    trig, _, _ = p.triggers()
    best = trig[np.argmax(trig["snr"])]
    assert int(best["sample"]) == j0
    assert abs(best["snr"] / 15.0 - 1) < 1e-5
    assert abs(best["phase"] - 0.3) < 4e-3


def test_ragged_window_valid_range_three_detectors_and_subset(mf):
    n, fs = 1 << 13, 512.0
    rng = np.random.default_rng(7)
    psd = synth.psd_bins(n, fs)
    m1, m2 = synth.sample_bank_uniform_masses(rng, 9, 1.4, 8.0)
    bank = np.stack([synth.taylorf2(n, fs, a, b, 25.0, dtype=np.complex64) for a, b in zip(m1, m2)])
    fd = np.stack([synth.coloured_noise_fd(rng, n, fs) for _ in range(3)])
    W, vb, ve = 500, 300, 7001
    p = _plan(mf, fs, n, 3, 25.0, 2.8, W, vb=vb, ve=ve, f_high=200.0)
    p.set_psd(psd)
    p.load_bank(torch.from_numpy(bank).to(DEV))
    dtil = fd.astype(np.complex64)
    sub = np.array([0, 2, 3, 7, 8], dtype=np.int32)
    p.filter(torch.from_numpy(dtil).to(DEV), subset=torch.from_numpy(sub).to(DEV))
    trig, _, _ = p.triggers()
    assert set(np.unique(trig["tmpl"])) <= set(sub.tolist())
    assert trig["sample"].min() >= vb and trig["sample"].max() < ve
    rho2, _ = oracle_rho2(dtil.astype(np.complex128), bank[sub], psd, n, fs, 25.0, 200.0)
    compare_triggers(trig, rho2, sub, 2.8, W, valid_begin=vb, valid_end=ve)


def test_empty_subset_zero_template_and_overflow(mf):
    n, fs = 1 << 12, 512.0
    rng = np.random.default_rng(9)
    psd = synth.psd_bins(n, fs)
    bank = np.stack([synth.taylorf2(n, fs, 3.0, 2.0, 30.0), np.zeros(n // 2 + 1)]).astype(np.complex64)
    fd = synth.coloured_noise_fd(rng, n, fs)[None].astype(np.complex64)
    p = _plan(mf, fs, n, 1, 30.0, 0.5, 64, max_trig=5)
    p.set_psd(psd)
    p.load_bank(bank)
    assert p.sigmasq()[1] == 0.0
    d = torch.from_numpy(fd).to(DEV)
    p.filter(d, subset=torch.zeros(0, dtype=torch.int32, device=DEV), n_subset=0)
    trig, n0, st = p.triggers()
    assert n0 == 0 and len(trig) == 0
    p.filter(d, subset=torch.tensor([1], dtype=torch.int32, device=DEV))
    assert p.triggers()[1] == 0  # all-zero template: sigma = 0, never a trigger
    p.filter(d)  # threshold 0.5: every window of template 0 has a peak -> 64 triggers, buffer of 5
    trig, nall, st = p.triggers(cap=100)
    assert nall == 64 and len(trig) == 5 and st == mf.MF_EOVERFLOW


def test_errors_are_reported_not_raised_in_c(mf):
    lib = mf.load()
    p = _plan(mf, 512.0, 4096, 1, 30.0, 5.0, 512)
    dt = torch.zeros((1, 2049), dtype=torch.complex64, device=DEV)
    assert lib.mf_filter(p.h, dt.data_ptr(), 2049, None, -1) == mf.MF_ESTATE
    assert b"PSD" in lib.mf_last_error(p.h)
    p.set_psd(synth.psd_bins(4096, 512.0))
    assert lib.mf_filter(p.h, dt.data_ptr(), 2049, None, -1) == mf.MF_ESTATE  # no bank
    p.load_bank(np.zeros((1, 2049), np.complex64))
    assert lib.mf_filter(p.h, dt.data_ptr(), 100, None, -1) == mf.MF_EINVAL
    assert lib.mf_filter(p.h, dt.data_ptr(), 2049, None, 3) == mf.MF_EINVAL  # null subset with a count
    with pytest.raises(mf.MFError):
        p.load_bank(np.zeros((1, 2049), np.complex64), dtype=mf.MF_F16)  # 16-bit bank without scales


def test_bounded_wait_timeout_is_reported_and_the_context_stays_usable(mf):
    """Failure detection without a fault: a wait that nothing completes gives up,
    every waiting thread returns, the plan reports MF_ETIMEOUT once, and the
    next filter gives the same triggers as before."""
    c = synth.make_config1()
    p = _plan(mf, c.fs, c.n, 1, c.f_low, c.thr, c.window)
    p.set_psd(c.psd)
    p.load_bank(torch.from_numpy(c.bank()).to(DEV))
    sfd = torch.from_numpy((c.noise_fd + c.signal_fd).astype(np.complex64)[None, :]).to(DEV)
    p.filter(sfd)
    ref, _, _ = p.triggers()
    assert p.selftest_wait() == 128
    with pytest.raises(mf.MFError) as e:
        p.triggers()
    assert e.value.status == mf.MF_ETIMEOUT
    p.filter(sfd)
    got, _, _ = p.triggers()
    assert np.array_equal(got, ref)


def test_template_range_shards_merge_to_the_unsharded_run(mf):
    """Multi-GPU layout by template range, run as shards on one GPU: the merged
    shard trigger lists equal the unsharded run exactly."""
    from paper_2309_00019_gb300.multi import merge_triggers

    c = synth.make_config1()
    p = _plan(mf, c.fs, c.n, 1, c.f_low, c.thr, c.window)
    p.set_psd(c.psd)
    p.load_bank(torch.from_numpy(c.bank()).to(DEV))
    sfd = torch.from_numpy((c.noise_fd + c.signal_fd).astype(np.complex64)[None, :]).to(DEV)
    p.filter(sfd)
    full, _, _ = p.triggers()
    parts = []
    for lo, hi in ((0, 21), (21, 40), (40, 64)):
        ids = torch.arange(lo, hi, dtype=torch.int32, device=DEV)
        p.filter(sfd, subset=ids)
        parts.append(p.triggers()[0].copy())
    assert np.array_equal(merge_triggers(parts), full)
