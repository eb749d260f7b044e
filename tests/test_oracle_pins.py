"""Pins of the FP64 oracle against things other than itself: closed forms,
statistics fixed by the mathematics, brute force on tiny inputs and the
numbers the paper prints.  All CPU."""

import math
import os

import numpy as np
import pytest
from scipy import stats

import synth
from oracle import mf_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.txt")


def golden():
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                out[k.strip()] = float(v)
    return out


# ---------------------------------------------------------------------------
# Eq. (1)-(2): noiseless injection recovers A * sigma exactly
# ---------------------------------------------------------------------------

def test_noiseless_injection_recovers_optimal_snr():
    c = synth.make_config1()
    bank = c.bank(np.complex128)
    w = O.weights(c.n, c.fs, c.f_low, c.f_high, c.psd)
    h = bank[c.inj_tmpl]
    sigma = math.sqrt(O.sigmasq(h, w))
    rho2, z = O.snr_squared(c.signal_fd, h, w, c.n)
    assert int(np.argmax(rho2)) == c.inj_sample
    assert math.sqrt(rho2[c.inj_sample]) == pytest.approx(c.inj_amp * sigma, rel=1e-12)
    # the injection was made at SNR 12 with a continuum norm: the discrete one agrees to 1e-3
    assert math.sqrt(rho2[c.inj_sample]) == pytest.approx(12.0, rel=1e-3)
    # phase of z at the peak is the injected phase (0 here)
    assert abs(math.atan2(z[c.inj_sample].imag, z[c.inj_sample].real)) < 1e-9


@pytest.mark.parametrize("phi0,j0", [(0.7, 123), (-2.5, 16000), (3.0, 0)])
def test_noiseless_injection_any_phase_and_time(phi0, j0):
    n, fs = 4096, 512.0
    psd = synth.psd_bins(n, fs)
    h = synth.taylorf2(n, fs, 3.0, 2.0, 30.0)
    k = np.arange(n // 2 + 1)
    A = 2.5e-21
    s = A * h * np.exp(-2j * math.pi * k * (j0 % n) / n) * np.exp(1j * phi0)
    w = O.weights(n, fs, 30.0, fs / 2, psd)
    rho2, z = O.snr_squared(s, h, w, n)
    sig = math.sqrt(O.sigmasq(h, w))
    assert int(np.argmax(rho2)) == j0 % n
    assert math.sqrt(rho2.max()) == pytest.approx(A * sig, rel=1e-12)
    ph = math.atan2(z[j0 % n].imag, z[j0 % n].real)
    assert math.cos(ph - phi0) == pytest.approx(1.0, abs=1e-12)


# ---------------------------------------------------------------------------
# Appendix A: in Gaussian noise rho^2 is chi^2 with 2 dof (mean 2, var 4)
# ---------------------------------------------------------------------------

def test_noise_rho2_is_chi2_two_dof():
    n, fs = 8192, 512.0
    psd = synth.psd_bins(n, fs)
    w = O.weights(n, fs, 30.0, fs / 2, psd)
    h = synth.taylorf2(n, fs, 5.0, 3.0, 30.0)
    p = w * np.abs(h) ** 2
    p = p / p.sum()
    R = 24
    rng = np.random.default_rng(11)
    means, at_fixed = [], []
    allr = []
    for _ in range(R):
        s = synth.coloured_noise_fd(rng, n, fs)
        rho2, _ = O.snr_squared(s, h, w, n)
        means.append(rho2.mean())
        at_fixed.append(rho2[::512])
        allr.append(rho2)
    # the mean over samples of one realisation has std 2 sqrt(sum p^2) (exponential |n_k|^2)
    sd = 2.0 * math.sqrt((p ** 2).sum()) / math.sqrt(R)
    assert abs(np.mean(means) - 2.0) < 5 * sd
    # per-sample distribution: Exp(mean 2), i.e. chi^2_2 (a dropped quadrature would give chi^2_1)
    x = np.concatenate(at_fixed)
    ks = stats.kstest(x, "expon", args=(0, 2.0))
    assert ks.pvalue > 1e-3
    v = np.concatenate(allr).var()
    assert v == pytest.approx(4.0, rel=0.15)


# ---------------------------------------------------------------------------
# brute force: O(N^2) time-domain correlation of the whitened analytic signals
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [16, 64, 128])
def test_bruteforce_time_domain_correlation(n):
    rng = np.random.default_rng(n)
    fs = 64.0
    nb = n // 2 + 1
    s = rng.standard_normal(nb) + 1j * rng.standard_normal(nb)
    h = rng.standard_normal(nb) + 1j * rng.standard_normal(nb)
    psd = rng.uniform(0.5, 2.0, nb)
    w = O.weights(n, fs, 3 * fs / n, fs / 2, psd)
    z = O.complex_snr(s, h, w, n)
    # direct sums, no FFT: analytic whitened series a(t), b(t), then circular correlation
    df = fs / n
    m = np.arange(n)
    a = np.zeros(n, complex)
    b = np.zeros(n, complex)
    for k in range(nb):
        if w[k] == 0:
            continue
        e = np.exp(2j * math.pi * m * k / n)
        a += s[k] / math.sqrt(psd[k]) * e
        b += h[k] / math.sqrt(psd[k]) * e
    zd = np.array([4 * df / n * sum(a[(mm + j) % n] * np.conj(b[mm]) for mm in range(n)) for j in range(n)])
    assert np.allclose(z, zd, rtol=1e-12, atol=1e-12 * np.abs(zd).max())


def test_band_excludes_dc_nyquist_and_bad_psd():
    n, fs = 64, 64.0
    psd = np.ones(n // 2 + 1)
    psd[5] = 0.0
    psd[6] = np.inf
    psd[7] = -1.0
    m = O.band_mask(n, fs, 0.0, fs / 2, psd)
    assert not m[0] and not m[n // 2]
    assert not m[5] and not m[6] and not m[7]
    assert m[1] and m[n // 2 - 1]
    m2 = O.band_mask(n, fs, 3.0, 10.0, psd)  # f_k = k Hz
    assert list(np.nonzero(m2)[0]) == [3, 4, 8, 9]


# ---------------------------------------------------------------------------
# Appendix A Eq. (9)-(10): max of N Rayleigh variables
# ---------------------------------------------------------------------------

def test_max_rayleigh_pdf_normalised_and_matches_simulation():
    for N in (1, 10, 1000):
        val = np.trapezoid(O.max_rayleigh_pdf(np.linspace(0, 12, 200001), N), dx=12 / 200000)
        assert val == pytest.approx(1.0, abs=1e-6)
    # the CDF derivative is the pdf
    r = np.linspace(0.5, 6, 50)
    eps = 1e-4
    d = (O.max_rayleigh_cdf(r + eps, 300) - O.max_rayleigh_cdf(r - eps, 300)) / (2 * eps)
    assert np.allclose(d, O.max_rayleigh_pdf(r, 300), rtol=1e-5, atol=1e-9)
    # Eq. (10) approaches Eq. (9) at large N in the tail
    rr = np.linspace(4.0, 6.0, 5)
    assert np.allclose(O.max_rayleigh_pdf_large_n(rr, 10 ** 5), O.max_rayleigh_pdf(rr, 10 ** 5), rtol=2e-3)
    # simulation: max of N independent Rayleigh variables
    rng = np.random.default_rng(5)
    N = 64
    x = np.sqrt(rng.standard_normal((20000, N)) ** 2 + rng.standard_normal((20000, N)) ** 2).max(1)
    ks = stats.kstest(x, lambda t: O.max_rayleigh_cdf(t, N))
    assert ks.pvalue > 1e-3


def test_window_maxima_in_noise_follow_eq9_with_effective_n():
    n, fs = 16384, 512.0
    psd = synth.psd_bins(n, fs)
    w = O.weights(n, fs, 30.0, fs / 2, psd)
    h = synth.taylorf2(n, fs, 6.0, 4.0, 30.0)
    rng = np.random.default_rng(3)
    mx = []
    for _ in range(12):
        s = synth.coloured_noise_fd(rng, n, fs)
        rho2, _ = O.snr_squared(s, h, w, n)
        mx.append(np.sqrt(rho2.reshape(-1, 512).max(1)))
    mx = np.concatenate(mx)
    # fit N_eff by maximum likelihood on a grid, then KS (App. A: N < N' samples are independent)
    grid = np.arange(20, 1024, 4)
    ll = [np.log(O.max_rayleigh_pdf(mx, N) + 1e-300).sum() for N in grid]
    neff = grid[int(np.argmax(ll))]
    assert 20 < neff <= 512
    ks = stats.kstest(mx, lambda t: O.max_rayleigh_cdf(t, neff))
    assert ks.pvalue > 1e-3


# ---------------------------------------------------------------------------
# threshold + clustering (Sec. II "peak >= rho_thr"), hand-made series
# ---------------------------------------------------------------------------

def test_cluster_windows_hand_made():
    r = np.zeros(20)
    r[1] = 16.0          # exactly thr^2 for thr 4: kept (inclusive)
    r[3] = 15.999999     # below
    r[6] = 20.0
    r[8] = 20.0          # tie with 6 in window [5,10): lowest index wins
    r[12] = 30.0
    r[17] = 1.0
    w, j, v = O.cluster_windows(r, 4.0, 5)
    assert list(w) == [0, 1, 2]
    assert list(j) == [1, 6, 12]
    assert list(v) == [16.0, 20.0, 30.0]
    # valid range cuts the first window and the tie partner
    w, j, v = O.cluster_windows(r, 4.0, 5, valid_begin=2, valid_end=7)
    assert list(j) == [6]


# ---------------------------------------------------------------------------
# decimation: FD truncation equals sampling a band-limited signal at the lower rate
# ---------------------------------------------------------------------------

def test_decimation_is_exact_for_band_limited_data():
    rng = np.random.default_rng(2)
    n2, fs2 = 4096, 2048.0
    nb = n2 // 2 + 1
    f = np.arange(nb) * fs2 / n2
    x = (rng.standard_normal(nb) + 1j * rng.standard_normal(nb)) * (f < 200.0)
    x[0] = 0
    s = synth.strain_from_fd(x, n2, fs2)
    lo = s[::4]
    s2 = O.strain_to_fd(s, fs2)
    s1 = O.decimate_fd(s2, n2 // 4)
    assert np.allclose(s1, O.strain_to_fd(lo, fs2 / 4), rtol=0, atol=1e-10 * np.abs(s1).max())


# ---------------------------------------------------------------------------
# coincidence with time shifts and the neighbourhood union (Sec. III)
# ---------------------------------------------------------------------------

def _trig(rows):
    return np.array([(d, t, s, r, 0.0) for d, t, s, r in rows], dtype=O.TRIGGER_DTYPE)


def test_coincidence_hand_made():
    R, sh, win = 1000, 100, 3
    trig = _trig([
        (0, 5, 10, 5.0),    # zero-lag partner at 12 (d = 2)
        (1, 5, 12, 4.0),
        (0, 5, 500, 6.0),   # shift k=2: 1-trigger at 300 -> 500 (d = 0)
        (1, 5, 300, 3.0),
        (0, 5, 998, 4.0),   # wraps: 1-trigger at 1 -> distance 3 on the ring at k=0
        (1, 5, 1, 4.0),
        (0, 7, 50, 9.0),    # other template: never pairs with template 5
        (1, 8, 50, 9.0),
    ])
    co = O.coincide(trig, 0, R, sh, 3, win)
    got = {(int(c["tmpl"]), int(c["shift"]), int(c["sample0"]), int(c["sample1"])) for c in co}
    assert (5, 0, 10, 12) in got
    assert (5, 2, 500, 300) in got
    assert (5, 0, 998, 1) in got
    assert all(t == 5 for t, _, _, _ in got)
    # brute force over every pair and shift (explicit loops)
    bf = set()
    for a in trig[trig["det"] == 0]:
        for b in trig[trig["det"] == 1]:
            if a["tmpl"] != b["tmpl"]:
                continue
            for k in range(4):
                s1 = (int(b["sample"]) + k * sh) % R
                d = abs(int(a["sample"]) - s1)
                if min(d, R - d) <= win:
                    bf.add((int(a["tmpl"]), k, int(a["sample"]), int(b["sample"])))
    assert got == bf
    rc = co[(co["sample0"] == 500)]["rho_c"][0]
    assert rc == pytest.approx(math.sqrt(36 + 9))
    assert list(O.followed_up(co, 7.0)) == []
    assert list(O.followed_up(co, 5.0)) == [5]


def test_nbhd_union_hand_made():
    ptr = np.array([0, 3, 3, 5, 7])
    idx = np.array([4, 1, 9, 2, 4, 9, 0], dtype=np.int32)
    assert list(O.nbhd_union([0, 2], ptr, idx)) == [1, 2, 4, 9]
    assert list(O.nbhd_union([1], ptr, idx)) == []
    assert list(O.nbhd_union([3, 1], ptr, idx)) == [0, 9]
    assert list(O.nbhd_union([], ptr, idx)) == []


# ---------------------------------------------------------------------------
# the template match behind the neighbourhood maps
# ---------------------------------------------------------------------------

def test_match_self_and_metric_neighbourhoods():
    n, fs = 2 ** 17, 2048.0
    psd = synth.psd_bins(n, fs)
    w = O.weights(n, fs, 30.0, fs / 2, psd)
    h = synth.taylorf2(n, fs, 8.0, 3.0, 30.0)
    assert O.match(h, h, w, n) == pytest.approx(1.0, abs=1e-12)
    hs = synth.taylorf2(n, fs, 8.0, 3.0, 30.0, t0=1.25, phi0=0.4)
    assert O.match(hs, h, w, n) == pytest.approx(1.0, abs=2e-3)  # sub-sample time offset
    # the quadratic-metric neighbourhood used by the banks tracks the exact match
    rng = np.random.default_rng(4)
    m1, m2, _, _ = synth.sample_bank_chirp_times(rng, 3000, 30.0, mc_lo=4.0, mc_hi=6.0)
    mm = synth.metric_match(m1[0], m2[0], m1, m2, 30.0, 30.0, fs / 2)
    sel = np.nonzero((mm > 0.92) & (mm < 0.999))[0][:4]
    assert len(sel) >= 2
    h0 = synth.taylorf2(n, fs, m1[0], m2[0], 30.0)
    for i in sel:
        ex = O.match(h0, synth.taylorf2(n, fs, m1[i], m2[i], 30.0), w, n)
        assert ex == pytest.approx(mm[i], abs=0.03)


# ---------------------------------------------------------------------------
# numbers the paper prints (Sec. V.C, Eq. 8; Table IV)
# ---------------------------------------------------------------------------

def test_cost_model_reproduces_printed_speedup():
    g = golden()
    sp = O.cost_model_speedup(g["nseg_H"], g["flat_templates"], g["coarse_templates"], g["stage2_templates_H"],
                              g["f_flat"], g["f_coarse"], g["t_seg"], gamma=1.0)
    assert sp == pytest.approx(g["speedup_mf_H"], abs=0.01)
    sp3 = O.cost_model_speedup(g["nseg_H"], g["flat_templates"], g["coarse_templates"], g["stage2_templates_H"],
                               g["f_flat"], g["f_coarse"], g["t_seg"], gamma=3.0)
    # printed 13.58 for "gamma ~ 3"; the model gives 13.50 at gamma = 3 exactly
    assert sp3 == pytest.approx(g["speedup_gamma3_H"], rel=0.01)
    # kappa cancels
    assert O.cost_model_speedup(g["nseg_H"], g["flat_templates"], g["coarse_templates"], g["stage2_templates_H"],
                                g["f_flat"], g["f_coarse"], g["t_seg"], gamma=1.0, kappa=7.0) == pytest.approx(sp)


def test_table_iv_ratios_and_gamma():
    g = golden()
    rH = g["corehours_flat_H"] / g["corehours_hier_bg_H"]
    rL = g["corehours_flat_L"] / g["corehours_hier_bg_L"]
    assert 14.0 <= rH <= 15.6 and 14.0 <= rL <= 15.6  # "14-15 times lower", Sec. V.C
    per_flat = g["block_flat_hours_H"] * 3600 / g["block_flat_applications"]
    per_nbhd = g["block_stage2_hours_H"] * 3600 / g["block_stage2_applications"]
    assert per_flat == pytest.approx(0.05, rel=0.15)
    assert per_nbhd == pytest.approx(0.15, rel=0.1)
    assert per_nbhd / per_flat == pytest.approx(3.0, rel=0.15)  # "approximately three times": 2.6
