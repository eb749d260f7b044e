"""Waveforms, noise, glitches and banks (inputs only; see the package header).

Conventions used throughout:
  * sampling rate fs, segment length N samples, dt = 1/fs, T = N*dt, df = 1/T;
  * one-sided frequency series on bins k = 0..N/2, f_k = k*df;
  * the Fourier convention x~[k] = dt * sum_j x[j] exp(-2*pi*i*j*k/N), so a
    signal that peaks at time t0 carries the factor exp(-2*pi*i*f*t0).
"""

from __future__ import annotations

import math

import numpy as np
from scipy import integrate

MTSUN_S = 4.925491025543576e-06  # G * M_sun / c^3 in seconds
EULER_GAMMA = 0.5772156649015329


# ---------------------------------------------------------------------------
# detector noise model
# ---------------------------------------------------------------------------

def psd_analytic(f):
    """Analytic one-sided PSD S_n(f) of the synthetic detectors.

    S_n = 1e-46 [x^-4.14 - 5 x^-2 + 111 (1 - x^2 + x^4/2) / (1 + x^2/2)],
    x = f / 215 Hz.  Positive for every f > 0 (minimum 3.3e-45 at 215 Hz).
    """
    f = np.asarray(f, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        x = f / 215.0
        s = 1e-46 * (x ** -4.14 - 5.0 * x ** -2 + 111.0 * (1.0 - x ** 2 + 0.5 * x ** 4) / (1.0 + 0.5 * x ** 2))
    return s


def psd_bins(n, fs):
    """PSD on the one-sided bins of an n-sample segment; bin 0 is set to 0.

    A zero (or any non-positive / non-finite) PSD bin means "no data here":
    both implementations give such bins zero weight.
    """
    k = np.arange(n // 2 + 1, dtype=np.float64)
    s = psd_analytic(k * fs / n)
    s[0] = 0.0
    return s


def coloured_noise_fd(rng, n, fs, f_gen_low=10.0, psd=psd_analytic):
    """Stationary Gaussian noise in the frequency domain.

    n~[k] = sqrt(T S_n(f_k) / 4) (a + i b), a, b ~ N(0, 1), so that
    E|n~[k]|^2 = T S_n / 2 (one-sided PSD convention).  Bins below
    ``f_gen_low`` (where the analytic PSD diverges), DC and Nyquist are zero.
    """
    T = n / fs
    nb = n // 2 + 1
    f = np.arange(nb) * fs / n
    a = rng.standard_normal(nb)
    b = rng.standard_normal(nb)
    keep = (f >= f_gen_low) & (np.arange(nb) < n // 2)
    amp = np.zeros(nb)
    amp[keep] = np.sqrt(T * psd(f[keep]) / 4.0)
    return amp * (a + 1j * b)


def strain_from_fd(xf, n, fs):
    """Time series whose one-sided spectrum (dt-normalised) is ``xf``."""
    return np.fft.irfft(np.asarray(xf), n=n) * fs


# ---------------------------------------------------------------------------
# compact-binary waveform: TaylorF2, 3.5PN non-spinning phase, Newtonian amplitude
# ---------------------------------------------------------------------------

def chirp_mass(m1, m2):
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    return (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2


def f_isco(m1, m2):
    """Schwarzschild ISCO gravitational-wave frequency 1/(6^1.5 pi M)."""
    M = (np.asarray(m1, dtype=np.float64) + np.asarray(m2, dtype=np.float64)) * MTSUN_S
    return 1.0 / (6.0 ** 1.5 * math.pi * M)


def chirp_times(m1, m2, f0):
    """Newtonian and 1.5PN chirp times (tau0, tau3) at reference frequency f0."""
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    M = (m1 + m2) * MTSUN_S
    eta = m1 * m2 / (m1 + m2) ** 2
    x = math.pi * M * f0
    tau0 = 5.0 / (256.0 * math.pi * f0 * eta) * x ** (-5.0 / 3.0)
    tau3 = 1.0 / (8.0 * f0 * eta) * x ** (-2.0 / 3.0)
    return tau0, tau3


def masses_from_chirp_times(tau0, tau3, f0):
    """Inverse of ``chirp_times``: (m1, m2) in solar masses with m1 >= m2.

    Returns NaN where (tau0, tau3) is unphysical (eta > 1/4).
    """
    tau0 = np.asarray(tau0, dtype=np.float64)
    tau3 = np.asarray(tau3, dtype=np.float64)
    x = 5.0 * tau3 / (32.0 * math.pi * tau0)  # pi M f0
    M = x / (math.pi * f0)
    eta = 1.0 / (8.0 * f0 * tau3) * x ** (-2.0 / 3.0)
    with np.errstate(invalid="ignore"):
        d = np.sqrt(1.0 - 4.0 * eta)
    mt = M / MTSUN_S
    m1 = 0.5 * mt * (1.0 + d)
    m2 = 0.5 * mt * (1.0 - d)
    bad = eta > 0.25
    m1 = np.where(bad, np.nan, m1)
    m2 = np.where(bad, np.nan, m2)
    return m1, m2


def duration_2pn(m1, m2, f_low):
    """Time from f_low to coalescence, post-Newtonian to 2PN order (seconds)."""
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    M = (m1 + m2) * MTSUN_S
    eta = m1 * m2 / (m1 + m2) ** 2
    v = (math.pi * M * f_low) ** (1.0 / 3.0)
    c2 = 4.0 / 3.0 * (743.0 / 336.0 + 11.0 / 4.0 * eta)
    c3 = -32.0 * math.pi / 5.0
    c4 = 2.0 * (3058673.0 / 1016064.0 + 5429.0 / 1008.0 * eta + 617.0 / 144.0 * eta ** 2)
    return 5.0 / (256.0 * eta) * M * v ** -8 * (1.0 + c2 * v ** 2 + c3 * v ** 3 + c4 * v ** 4)


def _pn_phase_coeffs(eta):
    """Non-spinning TaylorF2 phase coefficients psi_k (k = 0..7) and the two
    log coefficients (of ln v at v^5 and v^6), from the published 3.5PN
    stationary-phase expansion (Buonanno, Iyer, Ochsner, Pan, Sathyaprakash
    2009, Eq. 3.18)."""
    pi = math.pi
    p = [0.0] * 8
    p[0] = 1.0
    p[1] = 0.0
    p[2] = 20.0 / 9.0 * (743.0 / 336.0 + 11.0 / 4.0 * eta)
    p[3] = -16.0 * pi
    p[4] = 10.0 * (3058673.0 / 1016064.0 + 5429.0 / 1008.0 * eta + 617.0 / 144.0 * eta ** 2)
    p[5] = pi * (38645.0 / 756.0 - 65.0 / 9.0 * eta)
    p[6] = (11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi ** 2 - 6848.0 / 21.0 * EULER_GAMMA
            + eta * (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi ** 2)
            + 76055.0 / 1728.0 * eta ** 2 - 127825.0 / 1296.0 * eta ** 3
            - 6848.0 / 21.0 * math.log(4.0))
    p[7] = pi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta ** 2)
    log5 = 3.0 * p[5]          # coefficient of ln(v / v_lso) at v^5
    log6 = -6848.0 / 21.0      # coefficient of ln(v) at v^6
    return p, log5, log6


def taylorf2_phase(f, m1, m2):
    """Stationary-phase phase Psi(f) with t_c = phi_c = 0 (radians)."""
    f = np.asarray(f, dtype=np.float64)
    M = (m1 + m2) * MTSUN_S
    eta = m1 * m2 / (m1 + m2) ** 2
    p, log5, log6 = _pn_phase_coeffs(eta)
    v = np.cbrt(math.pi * M * f)
    vlso = 1.0 / math.sqrt(6.0)
    lv = np.log(v)
    s = p[0] + v * v * (p[2] + v * (p[3] + v * (p[4] + v * (
        p[5] + log5 * (lv - math.log(vlso))
        + v * (p[6] + log6 * lv + v * p[7])))))
    return -math.pi / 4.0 + 3.0 / (128.0 * eta * v ** 5) * s


def taylorf2(n, fs, m1, m2, f_low, t0=0.0, phi0=0.0, amp=1.0, dtype=np.complex128):
    """One-sided TaylorF2 template on the bins of an n-sample segment.

    h~(f) = amp f^{-7/6} exp(-i Psi(f)) exp(-2 pi i f t0) exp(i phi0) for
    f_low <= f <= f_ISCO (and below Nyquist), zero elsewhere.  With t0 = 0
    the merger sits at sample 0 and the inspiral wraps round the segment end.
    """
    nb = n // 2 + 1
    k = np.arange(nb)
    f = k * (fs / n)
    out = np.zeros(nb, dtype=np.complex128)
    fhi = min(float(f_isco(m1, m2)), fs / 2.0)
    sel = (f >= f_low) & (f <= fhi) & (k < n // 2)
    fs_ = f[sel]
    ph = taylorf2_phase(fs_, m1, m2) + 2.0 * math.pi * fs_ * t0 - phi0
    out[sel] = amp * fs_ ** (-7.0 / 6.0) * np.exp(-1j * ph)
    return out.astype(dtype)


def taylorf2_torch(n, fs, m1, m2, f_low, device, out=None, ld=None, block=32):
    """Same waveform as ``taylorf2`` for many templates at once, evaluated with
    torch in float64 on ``device`` and returned as complex64 rows [n_tmpl, ld]
    (ld >= n/2+1; columns outside each template's band are zero).  Used to fill
    multi-GB banks without a host round trip; numerically it matches
    ``taylorf2`` to float64 rounding before the final cast.  Templates are
    evaluated ``block`` at a time on the union of their bands."""
    import torch

    m1 = np.atleast_1d(np.asarray(m1, dtype=np.float64))
    m2 = np.atleast_1d(np.asarray(m2, dtype=np.float64))
    nb = n // 2 + 1
    ld = nb if ld is None else ld
    nt = len(m1)
    if out is None:
        out = torch.zeros((nt, ld), dtype=torch.complex64, device=device)
    else:
        out.zero_()
    lv_lso = math.log(1.0 / math.sqrt(6.0))
    M = (m1 + m2) * MTSUN_S
    eta = m1 * m2 / (m1 + m2) ** 2
    fhi = np.minimum(f_isco(m1, m2), fs / 2.0)
    k0 = int(math.ceil(f_low * n / fs - 1e-9))
    k1 = np.minimum(np.floor(fhi * n / fs + 1e-9).astype(np.int64), n // 2 - 1)
    for b0 in range(0, nt, block):
        b1 = min(nt, b0 + block)
        kmax = int(k1[b0:b1].max())
        if kmax < k0:
            continue
        ff = torch.arange(k0, kmax + 1, dtype=torch.float64, device=device) * (fs / n)
        coef = np.array([_pn_phase_coeffs(e) for e in eta[b0:b1]], dtype=object)
        P = torch.tensor(np.array([c[0] for c in coef], dtype=np.float64), device=device)  # [b, 8]
        L5 = torch.tensor(np.array([c[1] for c in coef], dtype=np.float64), device=device)[:, None]
        L6 = torch.tensor(np.array([c[2] for c in coef], dtype=np.float64), device=device)[:, None]
        Mb = torch.tensor(M[b0:b1], dtype=torch.float64, device=device)[:, None]
        eb = torch.tensor(eta[b0:b1], dtype=torch.float64, device=device)[:, None]
        v = torch.pow(math.pi * Mb * ff[None, :], 1.0 / 3.0)
        lv = torch.log(v)
        p = [P[:, i:i + 1] for i in range(8)]
        sv = p[0] + v * v * (p[2] + v * (p[3] + v * (p[4] + v * (
            p[5] + L5 * (lv - lv_lso) + v * (p[6] + L6 * lv + v * p[7])))))
        ph = -math.pi / 4.0 + 3.0 / (128.0 * eb * v ** 5) * sv
        a = ff[None, :] ** (-7.0 / 6.0)
        kk = torch.arange(k0, kmax + 1, device=device)[None, :]
        inband = kk <= torch.tensor(k1[b0:b1], device=device)[:, None]
        a = torch.where(inband, a, torch.zeros((), dtype=torch.float64, device=device))
        out[b0:b1, k0:kmax + 1] = torch.complex(a * torch.cos(ph), -a * torch.sin(ph)).to(torch.complex64)
    return out


def taylorf2_norm_continuum(m1, m2, f_low, f_high, psd=psd_analytic):
    """sqrt(4 int f^{-7/3} / S_n df) over [f_low, min(f_ISCO, f_high)] by
    adaptive quadrature of the continuous integral.  Only used to set injection
    amplitudes to a requested optimal SNR; the filters compute their own,
    discrete, normalisation."""
    fhi = min(float(f_isco(m1, m2)), f_high)
    val, _ = integrate.quad(lambda f: f ** (-7.0 / 3.0) / psd(f), f_low, fhi, limit=400)
    return math.sqrt(4.0 * val)


# ---------------------------------------------------------------------------
# glitches
# ---------------------------------------------------------------------------

def sine_gaussian(t, t0, f0, Q, amp, phi):
    """g(t) = amp exp(-(t-t0)^2/tau^2) sin(2 pi f0 (t-t0) + phi), tau = Q/(sqrt2 pi f0)."""
    tau = Q / (math.sqrt(2.0) * math.pi * f0)
    x = t - t0
    return amp * np.exp(-(x / tau) ** 2) * np.sin(2.0 * math.pi * f0 * x + phi)


def sine_gaussian_amplitude(snr, f0, Q, psd=psd_analytic):
    """Amplitude that gives a sine-Gaussian the requested optimal SNR in the
    narrow-band limit: rho^2 ~= amp^2 tau sqrt(pi/2) / S_n(f0)."""
    tau = Q / (math.sqrt(2.0) * math.pi * f0)
    return snr * math.sqrt(float(psd(f0)) / (tau * math.sqrt(math.pi / 2.0)))


# ---------------------------------------------------------------------------
# template banks
# ---------------------------------------------------------------------------

def sample_bank_uniform_masses(rng, n_tmpl, m_lo, m_hi):
    """Templates with component masses drawn uniformly in [m_lo, m_hi]
    (ordered m1 >= m2), kept in generation order."""
    a = rng.uniform(m_lo, m_hi, size=n_tmpl)
    b = rng.uniform(m_lo, m_hi, size=n_tmpl)
    return np.maximum(a, b), np.minimum(a, b)


def _in_region(m1, m2, mc_lo, mc_hi, m_min, m_max):
    mc = chirp_mass(m1, m2)
    ok = np.isfinite(m1) & np.isfinite(m2)
    with np.errstate(invalid="ignore"):
        ok &= (mc >= mc_lo) & (mc <= mc_hi) & (m2 >= m_min) & (m1 <= m_max)
    return ok


def sample_bank_chirp_times(rng, n_tmpl, f0, mc_lo=1.2, mc_hi=10.0, m_min=1.0, m_max=30.0):
    """Random bank, uniform in the chirp-time plane (tau0, tau3) at f0.

    The (tau0, tau3) plane is close to flat in the match metric, so uniform
    sampling there is a random bank of roughly even template density.  The
    region is chirp mass in [mc_lo, mc_hi], m2 >= m_min, m1 <= m_max.
    Returns (m1, m2, tau0, tau3) sorted by tau0 (descending duration), which
    makes template id order follow the bank geometry.
    """
    # bounding box of the region in (tau0, tau3) from a dense mass grid
    g = np.linspace(m_min, m_max, 600)
    A, B = np.meshgrid(g, g)
    sel = (A >= B) & _in_region(A, B, mc_lo, mc_hi, m_min, m_max)
    t0g, t3g = chirp_times(A[sel], B[sel], f0)
    lo0, hi0 = t0g.min(), t0g.max()
    lo3, hi3 = t3g.min(), t3g.max()
    m1s, m2s, t0s, t3s = [], [], [], []
    got = 0
    while got < n_tmpl:
        k = max(4 * (n_tmpl - got), 1024)
        t0 = rng.uniform(lo0, hi0, size=k)
        t3 = rng.uniform(lo3, hi3, size=k)
        m1, m2 = masses_from_chirp_times(t0, t3, f0)
        ok = _in_region(m1, m2, mc_lo, mc_hi, m_min, m_max)
        take = np.nonzero(ok)[0][: n_tmpl - got]
        m1s.append(m1[take]); m2s.append(m2[take]); t0s.append(t0[take]); t3s.append(t3[take])
        got += len(take)
    m1 = np.concatenate(m1s); m2 = np.concatenate(m2s)
    t0 = np.concatenate(t0s); t3 = np.concatenate(t3s)
    order = np.argsort(-t0, kind="stable")
    return m1[order], m2[order], t0[order], t3[order]


def _phase_metric(m1, m2, f0, f_low, f_high, psd=psd_analytic, nf=4000):
    """Match metric gamma_ij in (tau0, tau3) at one template, with t_c and
    phi_c maximised out (quadratic expansion of the match about the template).

    Moments J[x] = int x w df / int w df with w = f^{-7/3}/S_n on
    [f_low, min(f_ISCO, f_high)]; g_ab = (J[d_a Psi d_b Psi] - J[d_a Psi] J[d_b Psi]) / 2
    over (t_c, tau0, tau3), then t_c is projected out.  Phase derivatives are
    central differences of ``taylorf2_phase`` in (tau0, tau3).
    """
    fhi = min(float(f_isco(m1, m2)), f_high)
    f = np.geomspace(f_low, fhi, nf)
    w = f ** (-7.0 / 3.0) / psd(f)
    # trapezoid weights on the log grid
    dw = np.zeros_like(f)
    dw[1:] += 0.5 * np.diff(f)
    dw[:-1] += 0.5 * np.diff(f)
    w = w * dw
    w /= w.sum()
    t0, t3 = chirp_times(m1, m2, f0)
    h0, h3 = 1e-4 * t0, 1e-4 * t3

    def psi(a, b):
        x1, x2 = masses_from_chirp_times(a, b, f0)
        return taylorf2_phase(f, float(x1), float(x2))

    d0 = (psi(t0 + h0, t3) - psi(t0 - h0, t3)) / (2 * h0)
    d3 = (psi(t0, t3 + h3) - psi(t0, t3 - h3)) / (2 * h3)
    dt = 2.0 * math.pi * f
    D = [dt, d0, d3]
    J = np.array([(w * d).sum() for d in D])
    g = np.empty((3, 3))
    for a in range(3):
        for b in range(3):
            g[a, b] = 0.5 * ((w * D[a] * D[b]).sum() - J[a] * J[b])
    gam = g[1:, 1:] - np.outer(g[1:, 0], g[0, 1:]) / g[0, 0]
    return gam


def metric_match(c_m1, c_m2, f_m1, f_m2, f0, f_low, f_high, psd=psd_analytic):
    """Quadratic approximation 1 - gamma_ij dtau^i dtau^j of the match between
    template c and templates f (arrays), metric evaluated at c."""
    gam = _phase_metric(c_m1, c_m2, f0, f_low, f_high, psd)
    c0, c3 = chirp_times(c_m1, c_m2, f0)
    t0, t3 = chirp_times(f_m1, f_m2, f0)
    a = t0 - c0
    b = t3 - c3
    return 1.0 - (gam[0, 0] * a * a + 2 * gam[0, 1] * a * b + gam[1, 1] * b * b)


def nbhd_map(c_m1, c_m2, f_m1, f_m2, f0, f_low, f_high, min_match=0.9, max_size=2000, psd=psd_analytic):
    """Neighbourhood map coarse -> fine as CSR (ptr int64 [n_c+1], idx int32).

    nbhd(c) = fine templates whose metric match to c is >= min_match, ordered
    by decreasing match (ties: lower fine id first), truncated to max_size
    slots.  Also returns the matching match values (float64) per slot.
    """
    nc = len(c_m1)
    ptr = np.zeros(nc + 1, dtype=np.int64)
    idx_l, val_l = [], []
    ft0, ft3 = chirp_times(f_m1, f_m2, f0)
    for c in range(nc):
        gam = _phase_metric(c_m1[c], c_m2[c], f0, f_low, f_high, psd)
        c0, c3 = chirp_times(c_m1[c], c_m2[c], f0)
        a = ft0 - c0
        b = ft3 - c3
        m = 1.0 - (gam[0, 0] * a * a + 2 * gam[0, 1] * a * b + gam[1, 1] * b * b)
        sel = np.nonzero(m >= min_match)[0]
        order = np.lexsort((sel, -m[sel]))
        sel = sel[order][:max_size]
        idx_l.append(sel.astype(np.int32))
        val_l.append(m[sel])
        ptr[c + 1] = ptr[c] + len(sel)
    idx = np.concatenate(idx_l) if idx_l else np.zeros(0, np.int32)
    val = np.concatenate(val_l) if val_l else np.zeros(0)
    return ptr, idx, val


def taylorf2_chunks_torch(n, fs, m1, m2, f_low, device, chunk=128, ld=None):
    """Yield (row0, complex64 device tensor [rows, ld]) blocks of a TaylorF2 bank
    generated on ``device`` (see ``taylorf2_torch``); the tensor is reused."""
    import torch

    nb = n // 2 + 1
    ld = nb if ld is None else ld
    buf = None
    for r0 in range(0, len(m1), chunk):
        r1 = min(len(m1), r0 + chunk)
        if buf is None or buf.shape[0] != r1 - r0:
            buf = torch.zeros((r1 - r0, ld), dtype=torch.complex64, device=device)
        taylorf2_torch(n, fs, m1[r0:r1], m2[r0:r1], f_low, device, out=buf, ld=ld)
        torch.cuda.synchronize(device)
        yield r0, buf
