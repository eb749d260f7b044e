"""Pins of the oracle's Welch PSD estimate (CPU): it is the library routine
(scipy.signal.welch with the same window, overlap and averaging), the median
bias is the known alternating harmonic sum, and on coloured Gaussian noise the
estimate recovers the analytic PSD it was generated from."""

import math

import numpy as np
import pytest
from scipy import signal

import synth
from oracle import mf_oracle as O


@pytest.mark.parametrize("average", ["mean", "median"])
@pytest.mark.parametrize("seg_len,stride", [(1024, 512), (2048, 2048), (4096, 1024)])
def test_welch_equals_scipy(average, seg_len, stride):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 40000))
    got = O.psd_welch(x, 512.0, seg_len, stride, average)
    for d in range(2):
        f, ref = signal.welch(x[d], fs=512.0, window="hann", nperseg=seg_len, noverlap=seg_len - stride,
                              detrend=False, scaling="density", average=average)
        assert np.allclose(got[d], ref, rtol=1e-12, atol=0)


def test_median_bias_values():
    # n = 1, 2: no correction; n = 3: 1 - 1/2 + 1/3; large n -> ln 2
    assert O.median_bias(1) == 1.0 and O.median_bias(2) == 1.0
    assert O.median_bias(3) == pytest.approx(1 - 1 / 2 + 1 / 3)
    assert O.median_bias(4001) == pytest.approx(math.log(2.0), abs=2e-4)


def test_welch_recovers_the_analytic_psd():
    fs, n = 2048.0, 1 << 20
    rng = np.random.default_rng(1)
    x = synth.strain_from_fd(synth.coloured_noise_fd(rng, n, fs), n, fs)
    seg = 4096
    est = O.psd_welch(x, fs, seg, seg // 2, "median")[0]
    f = np.arange(seg // 2 + 1) * fs / seg
    band = (f >= 40) & (f <= 900)
    ratio = est[band] / synth.psd_analytic(f[band])
    # 511 half-overlapping segments: per-bin scatter ~7%, the band average within 1%
    assert abs(np.mean(ratio) - 1.0) < 0.01
    lo, hi = np.percentile(ratio, [1, 99])
    assert 0.8 < lo and hi < 1.2 and np.all(np.abs(ratio - 1.0) < 0.35)
