"""Pins of the oracle's overlapping-segment search (CPU): the segment cut
partitions the analysed data exactly once (brute force over every sample), and
an injection in long data is found at the same global sample and SNR whatever
the segment length, and as by one long filter over the whole data."""

import math

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O


@pytest.mark.parametrize("n_samples,tmpl_len,seg_len,window", [
    (32768, 2048, 4096, 512), (32768, 1500, 8192, 512), (30000, 4096, 8192, 512), (5000, 100, 4096, 64),
    (4096 * 3 + 7, 4096, 8192, 1024)])
def test_segments_partition_the_analysed_samples(n_samples, tmpl_len, seg_len, window):
    plan = O.segment_plan(n_samples, tmpl_len, seg_len, window)
    L = -(-tmpl_len // window) * window
    cover = np.zeros(n_samples, dtype=np.int64)
    for start, b, e in plan:
        assert start % window == 0 and 0 <= b < e <= seg_len and start + e <= n_samples
        assert b == L  # the first L samples of every segment wrap around and are not analysed
        cover[start + b:start + e] += 1
    assert np.all(cover[:L] == 0) and np.all(cover[L:] == 1)


def test_segment_too_short_is_rejected():
    with pytest.raises(ValueError):
        O.segment_plan(10000, 4000, 4096, 512)


def test_injection_found_at_same_global_time_for_every_segment_length():
    fs, f_low = 512.0, 30.0
    m1, m2 = 14.0, 11.0
    dur = synth.duration_2pn(m1, m2, f_low)
    assert dur < 3.0
    n_samples = 64 * 512
    n_big = 65536
    rng = np.random.default_rng(11)
    t0 = 37.3
    psd_big = synth.psd_bins(n_big, fs)
    w_big = O.weights(n_big, fs, f_low, fs / 2, psd_big)
    h_big = synth.taylorf2(n_big, fs, m1, m2, f_low)
    amp = 15.0 / math.sqrt(O.sigmasq(h_big, w_big))
    fd = synth.coloured_noise_fd(rng, n_big, fs) + synth.taylorf2(n_big, fs, m1, m2, f_low, t0=t0, amp=amp)
    strain = synth.strain_from_fd(fd, n_big, fs)[:n_samples]
    # one long filter of the zero-padded data (no wrap at the injection: t0 > duration)
    pad = np.zeros(n_big)
    pad[:n_samples] = strain
    r2, _ = O.snr_squared(O.strain_to_fd(pad, fs), h_big, w_big, n_big)
    j_ref = int(np.argmax(r2[:n_samples]))
    assert abs(j_ref - t0 * fs) <= 1
    found = []
    for seg_len in (4096, 8192, 16384):
        bank = synth.taylorf2(seg_len, fs, m1, m2, f_low)[None, :]
        trig = O.segmented_filter(strain[None, :], fs, synth.psd_bins(seg_len, fs), f_low, fs / 2, bank, seg_len,
                                  int(math.ceil(dur * fs)), 6.0, 512)
        near = trig[np.abs(trig["sample"] - j_ref) < 512]
        assert len(near) == 1
        found.append((int(near["sample"][0]), float(near["snr"][0])))
    for j, snr in found:
        assert abs(j - j_ref) <= 1
        assert snr == pytest.approx(math.sqrt(r2[j_ref]), rel=2e-3)
    # and the segment lengths with each other
    assert abs(found[1][1] - found[2][1]) / found[2][1] < 2e-3
