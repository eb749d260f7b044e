"""Pins of the oracle's chi^2 veto and re-weighted SNR (CPU): the band split
against brute force, closed forms of Eq. (4), chi^2 of an exactly matching
signal from the band powers alone, the chi^2 distribution with 2p - 2 degrees
of freedom in Gaussian noise, and a loud glitch that the veto down-weights."""

import math

import numpy as np
import pytest
from scipy import stats

import synth
from oracle import mf_oracle as O


def _setup(n=16384, fs=512.0, f_low=30.0, m=(1.6, 1.3)):
    psd = synth.psd_bins(n, fs)
    w = O.weights(n, fs, f_low, fs / 2, psd)
    h = synth.taylorf2(n, fs, m[0], m[1], f_low)
    return psd, w, h


def test_bands_split_the_power_evenly_and_match_brute_force():
    _, w, h = _setup()
    p = 16
    band = O.chisq_bins(h, w, p)
    pw = w * np.abs(h) ** 2
    s2 = pw.sum()
    # brute force: walk the bins, the band is the floor of p x (power strictly below) / total
    acc, ref = 0.0, np.full(len(h), -1)
    for k in range(len(h)):
        if w[k] > 0:
            ref[k] = min(int(p * acc / s2), p - 1)
        acc += pw[k]
    assert np.array_equal(band, ref)
    per = np.array([pw[band == l].sum() for l in range(p)]) / s2
    assert np.all(np.abs(per - 1 / p) < 0.02)  # each band holds ~1/p of sigma^2
    assert np.all(np.diff(band[band >= 0]) >= 0)  # contiguous, in frequency order


def test_newsnr_closed_forms():
    assert O.newsnr(10.0, 0.5) == 10.0
    assert O.newsnr(10.0, 1.0) == pytest.approx(10.0)
    assert O.newsnr(10.0, 3.0) == pytest.approx(10.0 / 14.0 ** (1 / 6))
    assert O.newsnr(8.0, 2.0) == pytest.approx(8.0 / 4.5 ** (1 / 6))
    assert O.reduced_chisq(30.0, 16) == 1.0


def test_exact_signal_chisq_is_the_band_power_imbalance():
    """s = A h shifted to j0: at j0, z_l = A P_l, so chi^2 = p A^2 sum (P_l - sigma^2/p)^2 / sigma^2."""
    n = 16384
    _, w, h = _setup(n)
    p, j0 = 16, 5000
    s2 = O.sigmasq(h, w)
    A = 20.0 / math.sqrt(s2)
    k = np.arange(len(h))
    s = A * h * np.exp(-2j * math.pi * k * j0 / n)
    band = O.chisq_bins(h, w, p)
    P = np.array([(w * np.abs(h) ** 2)[band == l].sum() for l in range(p)])
    expect = p * A * A * np.sum((P - s2 / p) ** 2) / s2
    assert O.chisq(s, h, w, n, j0, p) == pytest.approx(expect, rel=1e-9, abs=1e-12)
    assert expect < 0.1  # a matched signal passes the veto


def test_gaussian_noise_chisq_has_2p_minus_2_degrees_of_freedom():
    n, fs = 4096, 512.0
    p = 8
    _, w, h = _setup(n, fs, m=(5.0, 4.0))
    rng = np.random.default_rng(4)
    vals = []
    for _ in range(40):
        s = synth.coloured_noise_fd(rng, n, fs)
        for j in rng.integers(0, n, 10):
            vals.append(O.chisq(s, h, w, n, int(j), p))
    vals = np.array(vals)
    dof = 2 * p - 2
    assert abs(vals.mean() - dof) < 4 * math.sqrt(2 * dof / len(vals))
    assert stats.kstest(vals, stats.chi2(dof).cdf).pvalue > 1e-3


def test_glitch_is_down_weighted():
    """A loud sine-Gaussian seen by a chirp template: high chi^2_r, newsnr well below rho."""
    n, fs = 16384, 512.0
    p = 16
    psd, w, h = _setup(n, fs)
    rng = np.random.default_rng(5)
    t = np.arange(n) / fs
    a = synth.sine_gaussian_amplitude(150.0, 120.0, 8.0)
    g = synth.sine_gaussian(t, 16.0, 120.0, 8.0, a, 0.3)
    s = synth.coloured_noise_fd(rng, n, fs) + O.strain_to_fd(g, fs)
    rho2, _ = O.snr_squared(s, h, w, n)
    j = int(np.argmax(rho2))
    rho = math.sqrt(rho2[j])
    c = O.reduced_chisq(O.chisq(s, h, w, n, j, p), p)
    assert rho > 10 and c > 5
    assert O.newsnr(rho, c) < 0.6 * rho
