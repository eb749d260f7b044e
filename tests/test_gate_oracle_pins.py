"""Pins of the oracle's gating of loud short transients (CPU): the gate
statistic against a brute-force sum and against scipy's analytic signal of the
band-limited whitened strain, its chi^2_2 distribution in Gaussian noise, the
inverse Tukey window's closed forms, and a loud glitch that is found and
removed while a chirp elsewhere in the data keeps its SNR."""

import math

import numpy as np
import pytest
from scipy import signal, stats

import synth
from oracle import mf_oracle as O


def test_statistic_matches_brute_force_sum():
    n, fs, f_low, f_high = 64, 64.0, 5.0, 30.0
    rng = np.random.default_rng(0)
    psd = 1.0 + rng.uniform(0.0, 1.0, n // 2 + 1)
    s = rng.standard_normal(n // 2 + 1) + 1j * rng.standard_normal(n // 2 + 1)
    got = O.gate_statistic(s, psd, n, fs, f_low, f_high)[0]
    df = fs / n
    band = [k for k in range(1, n // 2) if f_low <= k * df < f_high]
    sig = math.sqrt(4 * df * len(band))
    for j in range(n):
        z = sum(4 * df * s[k] / math.sqrt(psd[k]) * complex(math.cos(2 * math.pi * j * k / n),
                                                             math.sin(2 * math.pi * j * k / n)) for k in band)
        assert got[j] == pytest.approx(abs(z) / sig, rel=1e-12, abs=1e-12)


def test_statistic_is_the_analytic_signal_envelope_of_the_whitened_strain():
    """|scipy.signal.hilbert(y)| of the band-limited whitened series y = irfft(s~ / sqrt(S_n))
    is (2 / N) |sum_band s~ / sqrt(S_n) e^{+2 pi i j k / N}|."""
    n, fs, f_low, f_high = 4096, 512.0, 20.0, 200.0
    psd = synth.psd_bins(n, fs)
    rng = np.random.default_rng(1)
    s = synth.coloured_noise_fd(rng, n, fs)
    m = O.band_mask(n, fs, f_low, f_high, psd)
    x = np.zeros(n // 2 + 1, dtype=np.complex128)
    x[m] = s[m] / np.sqrt(psd[m])
    env = np.abs(signal.hilbert(np.fft.irfft(x, n)))
    df = fs / n
    expect = env * (n / 2) * 4 * df / math.sqrt(4 * df * m.sum())
    assert np.allclose(O.gate_statistic(s, psd, n, fs, f_low, f_high)[0], expect, rtol=1e-9, atol=1e-12)


def test_statistic_is_chi2_with_two_dof_in_gaussian_noise():
    n, fs = 1 << 15, 1024.0
    psd = synth.psd_bins(n, fs)
    rng = np.random.default_rng(2)
    vals = []
    for _ in range(4):
        s = synth.coloured_noise_fd(rng, n, fs)
        vals.append(O.gate_statistic(s, psd, n, fs, 20.0, 500.0)[0] ** 2)
    v = np.concatenate(vals)
    assert abs(v.mean() - 2.0) < 0.05
    assert stats.kstest(v[::97], stats.chi2(2).cdf).pvalue > 1e-3  # thinned: neighbours are correlated


def test_window_closed_forms_and_product():
    n, fs, tz, tt = 4001, 100.0, 0.5, 1.0
    g = O.gate_window(n, fs, [2000], tz, tt)
    assert np.all(g[1950:2051] == 0.0)             # |t| <= t_zero
    assert g[2000 + 100] == pytest.approx(0.5)      # t_zero + t_taper / 2
    assert g[2000 - 100] == pytest.approx(0.5)
    assert np.all(g[:1850] == 1.0) and np.all(g[2151:] == 1.0)  # |t| >= t_zero + t_taper
    assert g[2000 + 75] == pytest.approx(0.5 * (1 - math.cos(math.pi * 0.25)))
    assert np.all(np.diff(g[2000:]) >= 0) and np.allclose(g[:2001], g[2000:][::-1])
    g2 = O.gate_window(n, fs, [2000, 2120], tz, tt)
    assert np.allclose(g2, g * O.gate_window(n, fs, [2120], tz, tt))
    assert g2[2160] == 0.0 and g2[2070] == 0.0  # inside the second gate's zero span
    assert g2[1880] == pytest.approx(0.5 * (1 - math.cos(math.pi * 0.7)))  # first gate's taper only


def test_loud_glitch_is_gated_and_a_chirp_elsewhere_keeps_its_snr():
    n, fs, f_low = 1 << 16, 1024.0, 20.0
    psd = synth.psd_bins(n, fs)
    rng = np.random.default_rng(3)
    t = np.arange(n) / fs
    noise = synth.strain_from_fd(synth.coloured_noise_fd(rng, n, fs), n, fs)
    a = synth.sine_gaussian_amplitude(400.0, 150.0, 6.0)  # a very loud, short transient
    glitch = synth.sine_gaussian(t, 20.0, 150.0, 6.0, a, 0.0)
    w = O.weights(n, fs, f_low, fs / 2, psd)
    h = synth.taylorf2(n, fs, 14.0, 11.0, f_low)
    assert synth.duration_2pn(14.0, 11.0, f_low) < 10.0  # the chirp stays clear of the gate at 20 s
    amp = 15.0 / math.sqrt(O.sigmasq(h, w))
    chirp = synth.strain_from_fd(synth.taylorf2(n, fs, 14.0, 11.0, f_low, t0=50.0, amp=amp), n, fs)
    x = noise + glitch + chirp
    rho_g = O.gate_statistic(O.strain_to_fd(x, fs), psd, n, fs, f_low, fs / 2)
    gates = O.gate_find(rho_g, 30.0, int(fs))
    assert len(gates) >= 1 and np.all(np.abs(gates["sample"] / fs - 20.0) < 0.1)
    assert rho_g[0][np.abs(t - 20.0) > 2.0].max() < 8.0  # only the glitch is that loud
    xg = O.gate_apply(x, fs, gates, 0.25, 0.25)
    assert np.all(xg[0][np.abs(t - gates["sample"][0] / fs) <= 0.25] == 0.0)
    after = O.gate_statistic(O.strain_to_fd(xg, fs), psd, n, fs, f_low, fs / 2)
    assert after.max() < 8.0
    # the chirp (45-50 s, far from the gate) keeps its SNR
    r_before, _ = O.snr_squared(O.strain_to_fd(noise + chirp, fs), h, w, n)
    r_after, _ = O.snr_squared(O.strain_to_fd(xg[0], fs), h, w, n)
    j0 = int(np.argmax(r_before))
    assert math.sqrt(r_after[j0]) == pytest.approx(math.sqrt(r_before[j0]), rel=0.02)
