"""Pins of the oracle's sine-Gaussian veto (CPU): the tile's spectrum against the
discrete transform of its time-domain form, the reduced statistic's mean of 1 in
Gaussian noise (where the re-weighting of Eq. 3 leaves every trigger alone), a
glitch in one tile that the veto cuts down, a chirp that it leaves alone, and the
values Eq. (3) fixes: rho^ = rho~ (chi^2_sg)^(-1/2) from chi^2_sg = 6 on,
inclusive, rho^ = rho~ below."""

import math

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O

OFFSETS = [15.0, 30.0, 45.0, 60.0, 75.0, 90.0, 105.0, 120.0]


def test_tile_is_the_spectrum_of_a_sine_gaussian():
    n, fs, f0, q = 1 << 14, 2048.0, 250.0, 20.0
    tau = q / (math.sqrt(2.0) * math.pi * f0)
    t = (np.arange(n) - n // 2) / fs
    x = np.exp(-(t / tau) ** 2) * np.cos(2 * math.pi * f0 * t)
    X = np.abs(np.fft.rfft(np.fft.ifftshift(x)))  # centred at t = 0: a real, even pulse
    g = O.sg_tile(n, fs, f0, q)
    m = g > 1e-6
    ratio = X[m] / g[m]
    assert np.allclose(ratio, ratio[np.argmax(g[m])], rtol=1e-6)  # the same Gaussian bump, up to a constant
    assert O.sg_tile(n, fs, f0, q)[int(round(f0 / (fs / n)))] == pytest.approx(1.0)


def test_reduced_statistic_has_mean_one_in_gaussian_noise():
    n, fs, f_low = 1 << 14, 2048.0, 30.0
    psd = synth.psd_bins(n, fs)
    w = O.weights(n, fs, f_low, fs / 2, psd)
    rng = np.random.default_rng(6)
    vals = []
    for _ in range(60):
        s = synth.coloured_noise_fd(rng, n, fs)
        for j in rng.integers(0, n, 5):
            c, used = O.sg_chisq(s, w, n, fs, int(j), 150.0, OFFSETS, 20.0, fs / 2)
            assert used == 8
            vals.append(c)
    v = np.array(vals)
    assert abs(v.mean() - 1.0) < 0.12  # 300 correlated-tile draws; each rho_l^2 / 2 has mean 1
    # on this scale Eq. (3)'s threshold of 6 is far in the noise tail, so Gaussian-noise triggers keep
    # rho~; the unreduced sum (2 n_used times larger, mean 16) would cross it in most draws
    assert v.max() < 6.0
    assert np.array_equal(O.sg_newsnr(np.full(v.shape, 5.0), v), np.full(v.shape, 5.0))
    assert np.mean(16.0 * v >= 6.0) > 0.9


def test_glitch_in_a_tile_is_cut_and_a_chirp_is_not():
    n, fs, f_low = 1 << 16, 2048.0, 30.0
    psd = synth.psd_bins(n, fs)
    w = O.weights(n, fs, f_low, fs / 2, psd)
    rng = np.random.default_rng(7)
    m1, m2 = 25.0, 20.0  # a heavy template: total mass above 30
    h = synth.taylorf2(n, fs, m1, m2, f_low)
    f_final = float(synth.f_isco(m1, m2))
    assert 60.0 < f_final < 150.0
    noise = synth.coloured_noise_fd(rng, n, fs)
    # a short broadband glitch (Q 3) at the template's final frequency: it rings the template and
    # puts power into the tiles above f_final, where the template has none
    t = np.arange(n) / fs
    a = synth.sine_gaussian_amplitude(60.0, f_final, 3.0)
    glitch = O.strain_to_fd(synth.sine_gaussian(t, 10.0, f_final, 3.0, a, 0.4), fs)
    r2, _ = O.snr_squared(noise + glitch, h, w, n)
    j = int(np.argmax(np.where(np.abs(t - 10.0) < 0.5, r2, 0.0)))
    rho = math.sqrt(r2[j])
    c, used = O.sg_chisq(noise + glitch, w, n, fs, j, f_final, OFFSETS, 20.0, fs / 2)
    assert used == 8 and rho > 15.0 and c > 20.0
    assert O.sg_newsnr(rho, c) < 0.3 * rho
    # the template's own chirp at SNR 12 in noise
    amp = 12.0 / math.sqrt(O.sigmasq(h, w))
    s = noise + synth.taylorf2(n, fs, m1, m2, f_low, t0=20.0, amp=amp)
    r2, _ = O.snr_squared(s, h, w, n)
    j = int(np.argmax(r2))
    c, _ = O.sg_chisq(s, w, n, fs, j, f_final, OFFSETS, 20.0, fs / 2)
    assert c < 6.0
    assert O.sg_newsnr(math.sqrt(r2[j]), c) == pytest.approx(math.sqrt(r2[j]))


def test_eq3_values_and_skipped_tiles():
    # Eq. (3): rho^ = rho~ (chi^2_sg)^(-1/2) if chi^2_sg >= 6, rho~ otherwise
    assert O.sg_newsnr(12.0, 9.0) == pytest.approx(4.0, rel=1e-15)  # chi^2_sg = 9: rho~ / 3
    assert O.sg_newsnr(10.0, 6.0) == pytest.approx(10.0 / math.sqrt(6.0), rel=1e-15)  # inclusive at 6
    below = np.nextafter(6.0, 0.0)
    assert O.sg_newsnr(10.0, below) == 10.0  # just below 6: untouched (the printed rule jumps at 6)
    for c in (0.0, 1.0, 4.0, 5.0, 5.999):
        assert O.sg_newsnr(7.5, c) == 7.5
    assert O.sg_newsnr(10.0, 100.0) == pytest.approx(1.0, rel=1e-15)
    r = np.array([3.5, 8.0, 20.0])
    assert np.allclose(O.sg_newsnr(r, np.array([6.25, 16.0, 400.0])), r / np.array([2.5, 4.0, 20.0]), rtol=1e-15)
    n, fs = 4096, 512.0
    w = O.weights(n, fs, 20.0, fs / 2, synth.psd_bins(n, fs))
    s = np.zeros(n // 2 + 1, dtype=np.complex128)
    c, used = O.sg_chisq(s, w, n, fs, 0, 200.0, OFFSETS, 20.0, fs / 2)
    assert used == 3 and c == 0.0  # 215, 230, 245 Hz are below 256 Hz; the rest are not
