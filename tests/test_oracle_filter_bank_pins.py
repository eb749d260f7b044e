"""Pin of the oracle's assembled filter (filter_bank: Eq. 1-2, the threshold and
the window clustering over every detector and template), on noiseless
injections whose triggers are known in closed form: which (det, tmpl, sample)
fire, rho = A sigma, the injected phase, and the subset / detector / valid-range
selections keeping the bank's own template ids."""

import math

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O

N, FS, F_LOW, W, THR = 8192, 512.0, 30.0, 512, 10.0
MASSES = [(1.4, 1.3), (9.0, 7.0), (30.0, 25.0)]  # mutual matches below 0.17


def _case():
    psd = synth.psd_bins(N, FS)
    w = O.weights(N, FS, F_LOW, FS / 2, psd)
    bank = np.stack([synth.taylorf2(N, FS, a, b, F_LOW) for a, b in MASSES])
    k = np.arange(N // 2 + 1)
    s = np.zeros((3, N // 2 + 1), dtype=np.complex128)
    # (det, tmpl, sample, SNR, phase): one circular injection A h e^{-2 pi i k j0 / N} e^{i phi} per
    # detector, so each row's own template sees exactly A sigma and the others stay below 0.17 of it
    inj = [(0, 2, 1000, 20.0, 0.0), (1, 0, 5000, 15.0, 0.7), (2, 1, 2000, 12.0, -1.2)]
    for d, t, j0, snr, phi in inj:
        a = snr / math.sqrt(O.sigmasq(bank[t], w))
        s[d] += a * bank[t] * np.exp(-2j * math.pi * k * j0 / N) * np.exp(1j * phi)
    return psd, bank, s, inj


def test_noiseless_injections_fire_exactly_their_own_windows():
    psd, bank, s, inj = _case()
    trig, s2 = O.filter_bank(s, bank, psd, N, FS, F_LOW, FS / 2, THR, W)
    assert [(int(t["det"]), int(t["tmpl"]), int(t["sample"])) for t in trig] == \
        sorted((d, t, j) for d, t, j, _, _ in inj)
    for t in trig:
        d, tm, j, snr, phi = next(x for x in inj if x[0] == t["det"] and x[1] == t["tmpl"])
        assert t["snr"] == pytest.approx(snr, rel=1e-9)
        assert math.remainder(t["phase"] - phi, 2 * math.pi) == pytest.approx(0.0, abs=1e-9)
    assert sorted(s2) == [0, 1, 2]


def test_subset_detectors_and_valid_range_keep_the_bank_ids():
    psd, bank, s, _ = _case()
    trig, _ = O.filter_bank(s, bank, psd, N, FS, F_LOW, FS / 2, THR, W, subset=[2, 0])
    assert [(int(t["det"]), int(t["tmpl"]), int(t["sample"])) for t in trig] == [(0, 2, 1000), (1, 0, 5000)]
    trig, _ = O.filter_bank(s, bank, psd, N, FS, F_LOW, FS / 2, THR, W, dets=[1, 2])
    assert [(int(t["det"]), int(t["tmpl"])) for t in trig] == [(1, 0), (2, 1)]
    trig, _ = O.filter_bank(s, bank, psd, N, FS, F_LOW, FS / 2, THR, W, valid_begin=1500, valid_end=6000)
    assert [(int(t["det"]), int(t["sample"])) for t in trig] == [(1, 5000), (2, 2000)]
    # a threshold above the loudest injection leaves nothing; one equal to an SNR keeps it (inclusive)
    assert len(O.filter_bank(s, bank, psd, N, FS, F_LOW, FS / 2, 20.0 + 1e-6, W)[0]) == 0
    trig, _ = O.filter_bank(s, bank, psd, N, FS, F_LOW, FS / 2, 15.0 * (1 - 1e-12), W)
    assert [(int(t["det"]), int(t["tmpl"])) for t in trig] == [(0, 2), (1, 0)]


def test_inner_product_closed_forms():
    psd, bank, _, _ = _case()
    w = O.weights(N, FS, F_LOW, FS / 2, psd)
    h = bank[1]
    assert O.inner(h, h, w) == pytest.approx(O.sigmasq(h, w), rel=1e-12)
    assert O.inner(h, 1j * h, w) == pytest.approx(0.0, abs=1e-12 * O.sigmasq(h, w))  # quadrature
    assert O.inner(bank[0], bank[2], w) == pytest.approx(O.inner(bank[2], bank[0], w), rel=1e-12)
    assert O.inner(2.0 * h, h, w) == pytest.approx(2.0 * O.sigmasq(h, w), rel=1e-12)


def test_hierarchy_follows_the_best_coarse_template_and_finds_the_injection():
    """A fine template injected at zero lag in both detectors (noiseless, SNR 12): its best-matching
    coarse template is followed, the stage-2 subset is the union of the followed neighbourhoods, and
    stage 2 fires the injected template at its sample with rho = 12."""
    n2, fs2, fs1, f_low = 8192, 512.0, 128.0, 20.0
    n1 = n2 // 4
    psd2, psd1 = synth.psd_bins(n2, fs2), synth.psd_bins(n1, fs1)
    fine_m = [(30, 28), (34, 30), (38, 33), (41, 35), (44, 38), (48, 42)]  # all below 76 Hz: stage 1 sees them whole
    coarse_m = [(31, 29), (40, 34), (47, 41)]
    fine = np.stack([synth.taylorf2(n2, fs2, a, b, f_low) for a, b in fine_m])
    coarse = np.stack([synth.taylorf2(n1, fs1, a, b, f_low) for a, b in coarse_m])
    ptr = np.array([0, 3, 5, 7])
    idx = np.array([0, 1, 2, 2, 3, 4, 5], dtype=np.int32)
    inj, j0 = 4, 3000
    w2 = O.weights(n2, fs2, f_low, fs2 / 2, psd2)
    k = np.arange(n2 // 2 + 1)
    fd = 12.0 / math.sqrt(O.sigmasq(fine[inj], w2)) * fine[inj] * np.exp(-2j * math.pi * k * j0 / n2)
    x = synth.strain_from_fd(fd, n2, fs2)
    strain = np.stack([x, x])
    r = O.hierarchical_search(strain, fs2, n2, fs1, psd1, psd2, coarse, fine, ptr, idx, f_low, 3.5, 4.0,
                              int(fs1), int(fs2), 2.0, 3, 0.015, 7.0)
    w1 = O.weights(n1, fs1, f_low, fs1 / 2, psd1)
    fine_at1 = synth.taylorf2(n1, fs1, *fine_m[inj], f_low)
    best = int(np.argmax([O.match(c, fine_at1, w1, n1) for c in coarse]))
    assert best == 2 and best in set(r["followed"].tolist())
    assert np.all(r["coinc"]["shift"] == 0)  # one trigger per detector: only zero lag pairs
    want = np.unique(np.concatenate([idx[ptr[c]:ptr[c + 1]] for c in r["followed"]]))
    assert np.array_equal(r["union"], want) and inj in set(r["union"].tolist())
    t2 = r["trig2"]
    hit = t2[(t2["tmpl"] == inj) & (t2["sample"] == j0)]
    assert sorted(hit["det"].tolist()) == [0, 1]
    assert np.allclose(hit["snr"], 12.0, rtol=1e-9)
