"""FP64 CPU oracle of the hierarchical matched-filter hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path and
imports nothing from it.

Every function is the plain definition written out with numpy in float64, in
the paper's order and notation.  The paper's statements it follows:

  * Eq. (2), Sec. II: noise-weighted inner product
        (x, y) = 4 Re int_{f_low}^{f_high} x~(f) y~*(f) / S_n(f) df
    discretised as 4 df sum_k over the analysis band.
  * Eq. (1), Sec. II and Appendix A: the SNR maximised over coalescence phase
    is the quadrature sum of the two orthogonal phases,
        rho(t_c) = |z(t_c)| / sigma,  z(t_c) = 4 df sum_k s~ h~* / S_n e^{+2 pi i f t_c},
        sigma^2 = (h, h).
  * Sec. V.C: all t_c of a segment at once by one inverse FFT per template.
  * Sec. II: a trigger is kept when the peak SNR is >= rho_thr (inclusive);
    Sec. III: rho_thr = 3.5 in stage 1 and 4 in stage 2.
  * Sec. III: stage 1 runs at 512 Hz, stage 2 at 2048 Hz on the union of the
    neighbourhoods of followed-up coarse templates; Sec. III / IV: coincident
    triggers are followed up including time-shifted (background) ones.
  * Appendix A, Eq. (9)-(10): distribution of the maximum of N Rayleigh
    variables (used by the tests to pin the noise statistics).
  * Sec. V.C, Eq. (8): the matched-filter cost model.

Readings where the paper is silent (the same readings the CUDA path takes):
  * band: bins k with f_low <= k df < f_high, k < N/2 (DC and Nyquist never
    used), and S_n[k] > 0 and finite;
  * clustering: fixed windows of W samples aligned to sample 0; one trigger
    per (detector, template, window) at the arg-max of rho^2 among samples that
    pass the threshold, ties to the lowest sample index;
  * decimation to a lower rate keeps the one-sided bins k <= N_out/2;
  * coincidence: same coarse template, circular distance of the sample indices
    (after shifting detector 1 by k * shift samples on the ring of analysed
    samples) <= window samples, network SNR sqrt(rho_0^2 + rho_1^2) as the
    ranking statistic, follow-up when it is >= the follow-up threshold.
"""

from __future__ import annotations

import math

import numpy as np

TRIGGER_DTYPE = np.dtype([("det", np.int32), ("tmpl", np.int32), ("sample", np.int64),
                          ("snr", np.float64), ("phase", np.float64)])
COINC_DTYPE = np.dtype([("tmpl", np.int32), ("shift", np.int32), ("sample0", np.int64),
                        ("sample1", np.int64), ("snr0", np.float64), ("snr1", np.float64),
                        ("rho_c", np.float64)])


# ---------------------------------------------------------------------------
# frequency-domain data and the analysis band (Eq. 2)
# ---------------------------------------------------------------------------

def strain_to_fd(strain, fs):
    """One-sided spectrum s~[k] = dt sum_j s[j] e^{-2 pi i j k / N}, k = 0..N/2."""
    s = np.asarray(strain, dtype=np.float64)
    return np.fft.rfft(s, axis=-1) / fs


def band_mask(n, fs, f_low, f_high, psd):
    """Bins entering every sum of Eq. (2): f_low <= f_k < f_high, 0 < k < N/2,
    PSD bin positive and finite."""
    nb = n // 2 + 1
    k = np.arange(nb)
    df = fs / n
    psd = np.asarray(psd, dtype=np.float64)
    ok = np.isfinite(psd) & (psd > 0)
    k_lo = int(math.ceil(f_low / df - 1e-9))
    k_hi = min(n // 2 - 1, int(math.ceil(f_high / df - 1e-9)) - 1)
    return ok & (k >= max(k_lo, 1)) & (k <= k_hi)


def weights(n, fs, f_low, f_high, psd):
    """w[k] = 4 df / S_n[k] on the band, 0 elsewhere (Eq. 2)."""
    m = band_mask(n, fs, f_low, f_high, psd)
    w = np.zeros(n // 2 + 1)
    w[m] = 4.0 * (fs / n) / np.asarray(psd, dtype=np.float64)[m]
    return w


def inner(x, y, w):
    """(x, y) = Re sum_k w[k] x[k] y*[k]  (Eq. 2, discretised)."""
    return float(np.real(np.sum(w * np.asarray(x) * np.conj(np.asarray(y)))))


def sigmasq(htilde, w):
    """sigma^2 = (h, h) for one template or a stack [n_tmpl, nbins]."""
    h = np.asarray(htilde)
    return np.sum(w * (h.real.astype(np.float64) ** 2 + h.imag.astype(np.float64) ** 2), axis=-1)


# ---------------------------------------------------------------------------
# the filter (Eq. 1 with Sec. V.C's FFT over t_c)
# ---------------------------------------------------------------------------

def complex_snr(stilde, htilde, w, n):
    """z[j] = sum_k w[k] s~[k] h~*[k] e^{+2 pi i j k / N}, j = 0..N-1 (circular).

    Negative-frequency bins are zero, so z is the complex (two-phase) filter
    output whose modulus is maximised over the coalescence phase.
    """
    x = np.zeros(n, dtype=np.complex128)
    nb = n // 2 + 1
    x[:nb] = w * np.asarray(stilde, dtype=np.complex128) * np.conj(np.asarray(htilde, dtype=np.complex128))
    return np.fft.ifft(x) * n


def snr_squared(stilde, htilde, w, n):
    """rho^2[j] = |z[j]|^2 / sigma^2 and z (Eq. 1, Appendix A)."""
    z = complex_snr(stilde, htilde, w, n)
    s2 = sigmasq(htilde, w)
    return (z.real ** 2 + z.imag ** 2) / s2, z


def cluster_windows(rho2, thr, window, valid_begin=0, valid_end=None):
    """Per-window peak among samples with rho^2 >= thr^2 (Sec. II "peak" reading).

    Returns (window index, sample index, rho^2) arrays, ordered by window.
    """
    rho2 = np.asarray(rho2, dtype=np.float64)
    n = len(rho2)
    valid_end = n if valid_end is None else valid_end
    thr2 = float(thr) * float(thr)
    out_w, out_j, out_r = [], [], []
    w_first = valid_begin // window
    w_last = (valid_end - 1) // window
    for wi in range(w_first, w_last + 1):
        a = max(wi * window, valid_begin)
        b = min((wi + 1) * window, valid_end)
        seg = rho2[a:b]
        ok = seg >= thr2
        if not ok.any():
            continue
        masked = np.where(ok, seg, -np.inf)
        j = int(np.argmax(masked))  # first index of the maximum
        out_w.append(wi); out_j.append(a + j); out_r.append(seg[j])
    return np.array(out_w, dtype=np.int64), np.array(out_j, dtype=np.int64), np.array(out_r)


def filter_bank(stilde, bank, psd, n, fs, f_low, f_high, thr, window,
                valid_begin=0, valid_end=None, subset=None, dets=None):
    """Triggers of every (detector, template) pair: Eq. (1)-(2) + threshold + clustering.

    stilde: complex [n_det, N/2+1]; bank: complex [n_tmpl, N/2+1].
    Returns a TRIGGER_DTYPE array sorted by (det, tmpl, sample) and sigma^2.
    """
    stilde = np.atleast_2d(np.asarray(stilde))
    w = weights(n, fs, f_low, f_high, psd)
    tmpl_ids = np.arange(len(bank)) if subset is None else np.asarray(subset)
    dets = range(stilde.shape[0]) if dets is None else dets
    recs = []
    s2_all = {}
    for d in dets:
        for t in tmpl_ids:
            h = np.asarray(bank[t])
            rho2, z = snr_squared(stilde[d], h, w, n)
            s2_all[int(t)] = sigmasq(h, w)
            _, js, r2 = cluster_windows(rho2, thr, window, valid_begin, valid_end)
            for j, r in zip(js, r2):
                recs.append((d, int(t), int(j), math.sqrt(r), math.atan2(z[j].imag, z[j].real)))
    trig = np.array(recs, dtype=TRIGGER_DTYPE)
    trig = np.sort(trig, order=["det", "tmpl", "sample"])
    return trig, s2_all


# ---------------------------------------------------------------------------
# PSD estimation upstream of the filter (the paper takes S_n from the data)
# ---------------------------------------------------------------------------

def median_bias(n):
    """Ratio of the median to the mean of n exponential periodogram values
    (FINDCHIRP, Allen et al., Appendix B): 1 - 1/2 + 1/3 - ... up to 1/(2m+1),
    m = (n - 1) // 2."""
    m = (n - 1) // 2
    return 1.0 + sum(1.0 / (2 * i + 1) - 1.0 / (2 * i) for i in range(1, m + 1))


def psd_welch(strain, fs, seg_len, stride, average="median"):
    """One-sided PSD of each row of strain by Welch's method: segments of
    seg_len samples every stride samples (those that fit), periodic Hann
    window w[j] = (1 - cos(2 pi j / seg_len)) / 2, no detrending,
    P[k] = c |sum_j w[j] x[j] e^{-2 pi i j k / n}|^2 / (fs sum_j w[j]^2) with
    c = 2 except at DC and Nyquist (c = 1); averaged over segments by the
    mean, or by the median divided by median_bias (reading: the paper does
    not describe its PSD estimate)."""
    x = np.atleast_2d(np.asarray(strain, dtype=np.float64))
    n_seg = (x.shape[1] - seg_len) // stride + 1
    j = np.arange(seg_len)
    w = 0.5 - 0.5 * np.cos(2 * math.pi * j / seg_len)
    out = np.zeros((x.shape[0], seg_len // 2 + 1))
    for d in range(x.shape[0]):
        per = np.empty((n_seg, seg_len // 2 + 1))
        for s in range(n_seg):
            X = np.fft.rfft(x[d, s * stride:s * stride + seg_len] * w)
            per[s] = np.abs(X) ** 2 / (fs * np.sum(w * w))
        per[:, 1:-1] *= 2.0
        out[d] = per.mean(axis=0) if average == "mean" else np.median(per, axis=0) / median_bias(n_seg)
    return out


# ---------------------------------------------------------------------------
# gating of loud short transients before the filter (Sec. VI; the paper cites
# the method without its statistic or parameters, so these are readings)
# ---------------------------------------------------------------------------

def gate_statistic(stilde, psd, n, fs, f_low, f_high):
    """rho_g[d, j] = |z_g[j]| / sigma_g, the envelope of the band-limited
    whitened strain in matched-filter SNR units:
        z_g[j] = 4 df sum_{k in band} s~[k] / sqrt(S_n[k]) e^{+2 pi i j k / N},
        sigma_g^2 = 4 df n_band
    (the band of Eq. 2).  In Gaussian noise rho_g^2 has mean 2 (two
    quadratures of unit variance)."""
    s = np.atleast_2d(np.asarray(stilde, dtype=np.complex128))
    m = band_mask(n, fs, f_low, f_high, psd)
    df = fs / n
    x = np.zeros((s.shape[0], n), dtype=np.complex128)
    x[:, :n // 2 + 1][:, m] = s[:, m] / np.sqrt(np.asarray(psd, dtype=np.float64)[m])
    z = 4.0 * df * n * np.fft.ifft(x, axis=-1)  # sum_k x[k] e^{+2 pi i j k / N}
    return np.abs(z) / math.sqrt(4.0 * df * int(m.sum()))


def gate_find(rho_g, thr, window, valid_begin=0, valid_end=None):
    """Gates: per row, the peak sample of every window of `window` samples
    that holds samples with rho_g >= thr (the filter's clustering rule,
    cluster_windows).  Returns a TRIGGER_DTYPE array (tmpl 0, phase 0)
    ordered by (det, sample)."""
    rows = []
    for d, r in enumerate(np.atleast_2d(rho_g)):
        _, j, r2 = cluster_windows(np.asarray(r, dtype=np.float64) ** 2, thr, window, valid_begin, valid_end)
        for jj, rr in zip(j, r2):
            rows.append((d, 0, int(jj), math.sqrt(rr), 0.0))
    return np.array(rows, dtype=TRIGGER_DTYPE)


def gate_window(n, fs, centers, t_zero, t_taper):
    """g[j] = product over gate centers c of the inverse Tukey window
    W(|j - c| / fs): W(t) = 0 for t <= t_zero, (1 - cos(pi (t - t_zero) /
    t_taper)) / 2 for t_zero < t < t_zero + t_taper, 1 beyond."""
    j = np.arange(n, dtype=np.float64)
    g = np.ones(n)
    for c in centers:
        t = np.abs(j - float(c)) / fs
        w = np.ones(n)
        w[t <= t_zero] = 0.0
        m = (t > t_zero) & (t < t_zero + t_taper)
        w[m] = 0.5 * (1.0 - np.cos(math.pi * (t[m] - t_zero) / t_taper))
        g *= w
    return g


def gate_apply(strain, fs, gates, t_zero, t_taper):
    """Gated strain: each row times gate_window of that row's gates."""
    x = np.array(np.atleast_2d(strain), dtype=np.float64)
    for d in range(x.shape[0]):
        c = gates["sample"][gates["det"] == d]
        if len(c):
            x[d] *= gate_window(x.shape[1], fs, c, t_zero, t_taper)
    return x


# ---------------------------------------------------------------------------
# signal-based veto at trigger times: chi^2_r and the re-weighted SNR (Eq. 4)
# ---------------------------------------------------------------------------

def chisq_bins(htilde, w, p):
    """Band edges of the chi^2 test: p contiguous bands of the analysis band,
    each holding ~1/p of the template power sigma^2 = sum w |h|^2.  Bin k goes
    to band floor(p C(k) / sigma^2), with C(k) the template power of the bins
    below k (reading; the paper cites the test, Eq. 4, without its bands).
    Returns an int array [N/2+1] of band indices (-1 outside the band)."""
    h = np.asarray(htilde, dtype=np.complex128)
    pw = w * (h.real ** 2 + h.imag ** 2)
    s2 = pw.sum()
    below = np.concatenate([[0.0], np.cumsum(pw)[:-1]])
    band = np.minimum(np.floor(p * below / s2).astype(np.int64), p - 1)
    band[w == 0] = -1
    return band


def chisq(stilde, htilde, w, n, sample, p):
    """Allen's chi^2 at one sample: the complex filter output z split by band,
    z_l = sum_{k in band l} w s~ h~* e^{+2 pi i k j / N}, and
    chi^2 = p sum_l |z_l - z / p|^2 / sigma^2 (2p - 2 degrees of freedom
    in Gaussian noise).  Returns chi^2."""
    h = np.asarray(htilde, dtype=np.complex128)
    s = np.asarray(stilde, dtype=np.complex128)
    band = chisq_bins(h, w, p)
    k = np.arange(len(h))
    terms = w * s * np.conj(h) * np.exp(2j * math.pi * k * int(sample) / n)
    z_l = np.array([terms[band == l].sum() for l in range(p)])
    z = z_l.sum()
    s2 = sigmasq(h, w)
    return float(p * np.sum(np.abs(z_l - z / p) ** 2) / s2)


def reduced_chisq(chi2, p):
    """chi^2_r = chi^2 / (2p - 2)."""
    return chi2 / (2 * p - 2)


def newsnr(rho, chi2_r):
    """Eq. (4): rho / [(1 + chi2_r^3) / 2]^(1/6) when chi2_r >= 1, else rho."""
    rho = np.asarray(rho, dtype=np.float64)
    c = np.asarray(chi2_r, dtype=np.float64)
    return np.where(c >= 1.0, rho / ((1.0 + c ** 3) / 2.0) ** (1.0 / 6.0), rho)


# ---------------------------------------------------------------------------
# sine-Gaussian veto of heavy templates (Sec. III: triggers of templates above
# 30 solar masses are further re-weighted with chi^2_sg; the paper cites the
# test without its tiles or normalisation, so these are readings)
# ---------------------------------------------------------------------------

def sg_tile(n, fs, f0, q):
    """One-sided spectrum of a sine-Gaussian tile of central frequency f0 and
    quality factor q: g~[k] = exp(-(pi tau (f_k - f0))^2), tau = q / (sqrt(2) pi f0)
    (the positive-frequency part of the transform of exp(-t^2 / tau^2) cos(2 pi f0 t),
    up to a constant), k = 0..N/2."""
    f = np.arange(n // 2 + 1) * (fs / n)
    tau = q / (math.sqrt(2.0) * math.pi * f0)
    return np.exp(-(math.pi * tau * (f - f0)) ** 2)


def sg_chisq(stilde, w, n, fs, sample, f_final, offsets, q, f_high):
    """Reduced sine-Gaussian chi^2 at one sample: tiles at f_l = f_final + offsets[l]
    (those below f_high), each with SNR rho_l = |sum_k w s~ g~_l e^{+2 pi i k j / N}| / sigma_l,
    sigma_l^2 = sum_k w g~_l^2, and chi2_r = sum_l rho_l^2 / (2 n_used) (mean 1 in Gaussian
    noise).  Returns (chi2_r, n_used)."""
    s = np.asarray(stilde, dtype=np.complex128)
    k = np.arange(n // 2 + 1)
    ph = np.exp(2j * math.pi * k * int(sample) / n)
    tot, used = 0.0, 0
    for off in offsets:
        f0 = float(f_final) + float(off)
        if f0 >= f_high:
            continue
        g = sg_tile(n, fs, f0, q)
        z = np.sum(w * s * g * ph)
        tot += abs(z) ** 2 / np.sum(w * g * g)
        used += 1
    return (tot / (2 * used) if used else 0.0), used


def sg_newsnr(newsnr_value, chi2_sg):
    """Eq. (3): rho^ = rho~ (chi2_sg)^(-1/2) when chi2_sg >= 6 (inclusive), else rho~.
    chi2_sg is the reduced statistic of sg_chisq (mean 1 in Gaussian noise)."""
    r = np.asarray(newsnr_value, dtype=np.float64)
    c = np.asarray(chi2_sg, dtype=np.float64)
    return np.where(c >= 6.0, r / np.sqrt(np.maximum(c, 6.0)), r)


# ---------------------------------------------------------------------------
# overlapping segments of long data (Sec. V.C)
# ---------------------------------------------------------------------------

def segment_plan(n_samples, tmpl_len, seg_len, window):
    """Overlapping segments of one template-length class (Sec. V.C analyses the
    data in overlapping segments; the cut is the reading below, the paper
    gives none).

    Templates last at most tmpl_len samples and are padded to seg_len.  In a
    segment the circular filter output at local sample j mixes in data from
    the segment's far end when j < template length, so the analysed part
    starts at L = tmpl_len rounded up to whole clustering windows.  Segments
    advance by stride = seg_len - L rounded down to whole windows (so
    windows never straddle two segments) and segment s analyses local
    samples [L, min(L + stride, n_samples - s stride)).  Data past the end are
    zero.  Returns [(start, begin, end)] in local sample units.
    """
    L = -(-int(tmpl_len) // window) * window
    stride = (seg_len - L) // window * window
    if stride <= 0:
        raise ValueError("segment too short for the template length")
    out = []
    s = 0
    while s * stride + L < n_samples:
        start = s * stride
        out.append((start, L, min(L + stride, n_samples - start)))
        s += 1
    return out


def segmented_filter(strain, fs, psd, f_low, f_high, bank, seg_len, tmpl_len, thr, window):
    """Triggers over long data: each overlapping segment of segment_plan is
    filtered as in filter_bank (Eq. 1-2) with its analysed range; samples are
    returned in global units.  strain [n_det, n_samples]; bank and psd on the
    segment's grid (seg_len / 2 + 1 bins)."""
    strain = np.atleast_2d(np.asarray(strain, dtype=np.float64))
    n_det, n_samples = strain.shape
    recs = []
    for start, b, e in segment_plan(n_samples, tmpl_len, seg_len, window):
        seg = np.zeros((n_det, seg_len))
        take = min(seg_len, n_samples - start)
        seg[:, :take] = strain[:, start:start + take]
        trig, _ = filter_bank(strain_to_fd(seg, fs), bank, psd, seg_len, fs, f_low, f_high, thr, window,
                              valid_begin=b, valid_end=e)
        trig["sample"] += start
        recs.append(trig)
    trig = np.concatenate(recs) if recs else np.zeros(0, TRIGGER_DTYPE)
    return np.sort(trig, order=["det", "tmpl", "sample"])


# ---------------------------------------------------------------------------
# hierarchy glue (Sec. III)
# ---------------------------------------------------------------------------

def decimate_fd(stilde, n_out):
    """Spectrum of the same data at a lower rate: keep bins k <= n_out/2."""
    return np.asarray(stilde)[..., : n_out // 2 + 1].copy()


def coincide(trig, ring_begin, ring_end, shift_samples, n_shifts, window_samples, rho_c_thr=None):
    """Two-detector coincidences, zero-lag (k = 0) and time-shifted (k >= 1).

    A detector-0 trigger at s0 and a detector-1 trigger at s1 of the same
    template are coincident at shift k when the circular distance of s0 and
    s1 + k * shift_samples on the ring [ring_begin, ring_end) is at most
    window_samples.  rho_c = sqrt(rho_0^2 + rho_1^2).  Optionally keeps only
    rho_c >= rho_c_thr.  Sorted by (tmpl, shift, sample0).
    """
    R = ring_end - ring_begin
    t0 = trig[trig["det"] == 0]
    t1 = trig[trig["det"] == 1]
    out = []
    for tm in np.unique(np.concatenate([t0["tmpl"], t1["tmpl"]])):
        a = t0[t0["tmpl"] == tm]
        b = t1[t1["tmpl"] == tm]
        if len(a) == 0 or len(b) == 0:
            continue
        for k in range(n_shifts + 1):
            sb = (b["sample"] - ring_begin + k * shift_samples) % R
            sa = a["sample"] - ring_begin
            d = (sa[:, None] - sb[None, :]) % R
            d = np.minimum(d, R - d)
            ia, ib = np.nonzero(d <= window_samples)
            for i, j in zip(ia, ib):
                rc = math.sqrt(a["snr"][i] ** 2 + b["snr"][j] ** 2)
                if rho_c_thr is not None and rc < rho_c_thr:
                    continue
                out.append((tm, k, a["sample"][i], b["sample"][j], a["snr"][i], b["snr"][j], rc))
    c = np.array(out, dtype=COINC_DTYPE)
    return np.sort(c, order=["tmpl", "shift", "sample0", "sample1"])


def followed_up(coincs, rho_c_thr):
    """Coarse template ids with at least one coincidence (any shift) of rho_c >= thr."""
    sel = coincs["rho_c"] >= rho_c_thr
    return np.unique(coincs["tmpl"][sel]).astype(np.int32)


def background_count(stat_bg, x, scale=1.0):
    """n_b(x): background coincidences with statistic >= x, times scale (the
    ratio of background volumes, Sec. IV: the hierarchical background is
    scaled by the ratio of time-shift intervals)."""
    bg = np.sort(np.asarray(stat_bg, dtype=np.float64))
    x = np.asarray(x, dtype=np.float64)
    return scale * (len(bg) - np.searchsorted(bg, x, side="left"))


def far_count(stat_fg, stat_bg, t_bg, scale=1.0):
    """Eq. (6): FAR = (1 + n_b(Lambda_b >= Lambda_f)) / T_b for each foreground value."""
    return (1.0 + background_count(stat_bg, stat_fg, scale)) / float(t_bg)


def tail_fit(stat_bg, fit_min, scale=1.0):
    """Sec. IV: least-squares line log n_b = alpha + beta Lambda through the
    cumulative background counts at every background value >= fit_min
    (natural logarithm; n_b scaled as in background_count).  Returns (alpha, beta)."""
    bg = np.sort(np.asarray(stat_bg, dtype=np.float64))
    x = bg[bg >= fit_min]
    if len(x) < 2:
        raise ValueError("fewer than two background values above fit_min")
    y = np.log(background_count(bg, x, scale))
    A = np.stack([np.ones_like(x), x], axis=1)
    (alpha, beta), *_ = np.linalg.lstsq(A, y, rcond=None)
    return float(alpha), float(beta)


def far_fit(stat_fg, alpha, beta, t_bg):
    """Eq. (6) with the fitted background: (1 + exp(alpha + beta Lambda_f)) / T_b."""
    return (1.0 + np.exp(alpha + beta * np.asarray(stat_fg, dtype=np.float64))) / float(t_bg)


def nbhd_union(coarse_ids, ptr, idx):
    """Union of the neighbourhoods of the followed-up coarse templates (Sec. III),
    as sorted unique fine-template ids."""
    parts = [np.asarray(idx[ptr[c]:ptr[c + 1]]) for c in coarse_ids]
    if not parts:
        return np.zeros(0, dtype=np.int32)
    return np.unique(np.concatenate(parts)).astype(np.int32)


def hierarchical_search(strain, fs2, n2, fs1, psd1, psd2, coarse, fine, ptr, idx, f_low,
                        thr1, thr2, window1, window2, shift_s, n_shifts, coinc_s, rho_c_thr,
                        f_high1=None, f_high2=None, fine_subset_cap=None):
    """Both stages of Sec. III on one segment of two-detector strain.

    Stage 1: decimate to fs1, filter the coarse bank, threshold thr1.
    Coincidences (zero-lag and time-shifted); follow up coarse templates with
    rho_c >= rho_c_thr.  Stage 2: filter the union of their neighbourhoods at
    fs2, threshold thr2.  Returns a dict of every intermediate result.
    """
    n1 = int(round(n2 * fs1 / fs2))
    f_high1 = fs1 / 2 if f_high1 is None else f_high1
    f_high2 = fs2 / 2 if f_high2 is None else f_high2
    s2 = strain_to_fd(strain, fs2)
    s1 = decimate_fd(s2, n1)
    trig1, _ = filter_bank(s1, coarse, psd1, n1, fs1, f_low, f_high1, thr1, window1)
    co = coincide(trig1, 0, n1, int(round(shift_s * fs1)), n_shifts, int(math.floor(coinc_s * fs1 + 1e-9)))
    fu = followed_up(co, rho_c_thr)
    union = nbhd_union(fu, ptr, idx)
    trig2, _ = filter_bank(s2, fine, psd2, n2, fs2, f_low, f_high2, thr2, window2, subset=union)
    return dict(stilde2=s2, stilde1=s1, trig1=trig1, coinc=co, followed=fu, union=union, trig2=trig2)


# ---------------------------------------------------------------------------
# template match (neighbourhood definition) and paper formulas used as pins
# ---------------------------------------------------------------------------

def match(h1, h2, w, n):
    """max over t_c and phase of (h1, h2(t_c)) / (sigma_1 sigma_2)."""
    z = complex_snr(h1, h2, w, n)
    return float(np.abs(z).max() / math.sqrt(sigmasq(h1, w) * sigmasq(h2, w)))


def max_rayleigh_pdf(rho, N):
    """Eq. (9): pdf of the largest of N independent unit Rayleigh variables."""
    rho = np.asarray(rho, dtype=np.float64)
    e = np.exp(-rho ** 2 / 2.0)
    return N * rho * e * (1.0 - e) ** (N - 1)


def max_rayleigh_pdf_large_n(rho, N):
    """Eq. (10): large-N form N rho exp(-(rho^2/2 + N e^{-rho^2/2}))."""
    rho = np.asarray(rho, dtype=np.float64)
    return N * rho * np.exp(-(rho ** 2 / 2.0 + N * np.exp(-rho ** 2 / 2.0)))


def max_rayleigh_cdf(rho, N):
    """CDF of Eq. (9): (1 - e^{-rho^2/2})^N."""
    rho = np.asarray(rho, dtype=np.float64)
    return (1.0 - np.exp(-rho ** 2 / 2.0)) ** N


def cost_model_speedup(n_seg, n_flat, n_stage1, n_stage2, f_flat, f_coarse, t_seg, gamma, kappa=1.0):
    """Eq. (8): speed-up of the hierarchical over the flat matched filtering,
    O = kappa f t log(f t), O_fine = gamma O_flat."""
    o_flat = kappa * f_flat * t_seg * math.log(f_flat * t_seg)
    o_coarse = kappa * f_coarse * t_seg * math.log(f_coarse * t_seg)
    o_fine = gamma * o_flat
    return n_seg * n_flat * o_flat / (n_seg * n_stage1 * o_coarse + n_stage2 * o_fine)
