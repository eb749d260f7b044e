"""The synthetic workloads (inputs only).

make_config1: one detector, 32 s at 512 Hz (N = 16384), 64 TaylorF2 templates
    with m1, m2 ~ U(1.4, 10), template 17 injected (circularly, at sample N/2)
    at optimal SNR 12, threshold 5.5, 1 s clustering windows.
make_config2: two detectors, 512 s at 2048 Hz (N = 2^20), 20 sine-Gaussian
    glitches per detector, 50 TaylorF2 injections at SNR 6-20, a 2,000-template
    coarse bank for stage 1 at 512 Hz and a 20,000-template fine bank for
    stage 2 at 2048 Hz with its neighbourhood map (match >= 0.9).
    ``small=True`` gives a scaled-down copy (32 s, 48 coarse, 480 fine) with
    the same structure, for tests the oracle finishes in seconds.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import generators as g


@dataclass
class Config1:
    n: int
    fs: float
    f_low: float
    f_high: float
    thr: float
    window: int
    psd: np.ndarray
    m1: np.ndarray
    m2: np.ndarray
    inj_tmpl: int
    inj_snr: float
    inj_sample: int
    inj_amp: float
    noise_fd: np.ndarray          # complex128 [N/2+1]
    signal_fd: np.ndarray         # complex128 [N/2+1], the injected signal alone
    strain: np.ndarray            # float32 [1, N]

    def bank(self, dtype=np.complex64):
        return np.stack([g.taylorf2(self.n, self.fs, a, b, self.f_low, dtype=dtype)
                         for a, b in zip(self.m1, self.m2)])


def make_config1(seed=0, n=16384, fs=512.0, n_tmpl=64, inj_tmpl=17, inj_snr=12.0,
                 f_low=30.0, thr=5.5):
    rng = np.random.default_rng(seed)
    noise = g.coloured_noise_fd(rng, n, fs)
    m1, m2 = g.sample_bank_uniform_masses(rng, n_tmpl, 1.4, 10.0)
    j0 = n // 2
    amp = inj_snr / g.taylorf2_norm_continuum(m1[inj_tmpl], m2[inj_tmpl], f_low, fs / 2)
    h = g.taylorf2(n, fs, m1[inj_tmpl], m2[inj_tmpl], f_low)
    k = np.arange(n // 2 + 1)
    sig = amp * h * np.exp(-2j * math.pi * k * j0 / n)
    strain = g.strain_from_fd(noise + sig, n, fs).astype(np.float32)[None, :]
    return Config1(n=n, fs=fs, f_low=f_low, f_high=fs / 2, thr=thr, window=int(round(fs)),
                   psd=g.psd_bins(n, fs), m1=m1, m2=m2, inj_tmpl=inj_tmpl, inj_snr=inj_snr,
                   inj_sample=j0, inj_amp=amp, noise_fd=noise, signal_fd=sig, strain=strain)


@dataclass
class Config2:
    n2: int
    fs2: float
    n1: int
    fs1: float
    f_low: float
    thr1: float
    thr2: float
    window1: int
    window2: int
    shift_s: float
    n_shifts: int
    coinc_s: float
    rho_c_thr: float
    psd1: np.ndarray
    psd2: np.ndarray
    coarse_m1: np.ndarray
    coarse_m2: np.ndarray
    fine_m1: np.ndarray
    fine_m2: np.ndarray
    nbhd_ptr: np.ndarray
    nbhd_idx: np.ndarray
    nbhd_match: np.ndarray
    strain: np.ndarray            # float32 [2, n2]
    injections: dict = field(default_factory=dict)
    glitches: dict = field(default_factory=dict)

    def coarse_bank(self, ids=None, dtype=np.complex64):
        ids = range(len(self.coarse_m1)) if ids is None else ids
        return np.stack([g.taylorf2(self.n1, self.fs1, self.coarse_m1[i], self.coarse_m2[i], self.f_low,
                                    dtype=dtype) for i in ids])

    def fine_bank(self, ids=None, dtype=np.complex64):
        ids = range(len(self.fine_m1)) if ids is None else ids
        return np.stack([g.taylorf2(self.n2, self.fs2, self.fine_m1[i], self.fine_m2[i], self.f_low,
                                    dtype=dtype) for i in ids])


def _banks(rng, n_coarse, n_fine, f_low, f_high, min_match):
    cm1, cm2, _, _ = g.sample_bank_chirp_times(rng, n_coarse, f_low)
    fm1, fm2, _, _ = g.sample_bank_chirp_times(rng, n_fine, f_low)
    ptr, idx, val = g.nbhd_map(cm1, cm2, fm1, fm2, f_low, f_low, f_high, min_match=min_match)
    return cm1, cm2, fm1, fm2, ptr, idx, val


def make_banks(seed=1, n_coarse=2000, n_fine=20000, f_low=30.0, f_high=1024.0, min_match=0.9):
    """The coarse and fine banks and neighbourhood map of the two-stage workload
    alone (the same draws as make_config2 with the same seed):
    (coarse m1, m2, fine m1, m2, nbhd ptr, nbhd idx, nbhd match)."""
    return _banks(np.random.default_rng(seed), n_coarse, n_fine, f_low, f_high, min_match)


def make_config2(seed=1, small=False):
    if small:
        T, n_coarse, n_fine, n_glitch, n_inj, n_shifts, min_match = 32.0, 48, 480, 4, 4, 5, 0.5
    else:
        T, n_coarse, n_fine, n_glitch, n_inj, n_shifts, min_match = 512.0, 2000, 20000, 20, 50, 101, 0.9
    fs2, fs1, f_low = 2048.0, 512.0, 30.0
    n2 = int(T * fs2)
    n1 = int(T * fs1)
    rng = np.random.default_rng(seed)
    # banks: random in the chirp-time plane, chirp mass 1.2-10
    cm1, cm2, fm1, fm2, ptr, idx, val = _banks(rng, n_coarse, n_fine, f_low, fs2 / 2, min_match)
    # noise
    nb = n2 // 2 + 1
    fd = np.stack([g.coloured_noise_fd(rng, n2, fs2) for _ in range(2)])
    # injections (same optimal SNR in both detectors, independent phases, dt_HL within 10 ms)
    im1, im2, _, _ = g.sample_bank_chirp_times(rng, n_inj, f_low)
    snr = rng.uniform(6.0, 20.0, n_inj)
    slot = T / n_inj
    tc = (np.arange(n_inj) + 0.5) * slot + rng.uniform(-0.25, 0.25, n_inj) * slot
    dt_hl = rng.uniform(-0.010, 0.010, n_inj)
    phi = rng.uniform(0, 2 * math.pi, (n_inj, 2))
    amp = np.array([snr[i] / g.taylorf2_norm_continuum(im1[i], im2[i], f_low, fs2 / 2) for i in range(n_inj)])
    for i in range(n_inj):
        for d in range(2):
            t0 = tc[i] + (dt_hl[i] if d == 1 else 0.0)
            fd[d] += g.taylorf2(n2, fs2, im1[i], im2[i], f_low, t0=t0, phi0=phi[i, d], amp=amp[i])
    strain = np.stack([g.strain_from_fd(fd[d], n2, fs2) for d in range(2)])
    # glitches (time domain)
    t = np.arange(n2) / fs2
    gl = dict(det=[], t0=[], f0=[], Q=[], snr=[])
    for d in range(2):
        for _ in range(n_glitch):
            f0 = rng.uniform(30.0, 500.0)
            Q = rng.uniform(5.0, 20.0)
            s = rng.uniform(8.0, 50.0)
            t0 = rng.uniform(1.0, T - 1.0)
            ph = rng.uniform(0, 2 * math.pi)
            a = g.sine_gaussian_amplitude(s, f0, Q)
            tau = Q / (math.sqrt(2.0) * math.pi * f0)
            lo = max(0, int((t0 - 6 * tau) * fs2))
            hi = min(n2, int((t0 + 6 * tau) * fs2) + 1)
            strain[d, lo:hi] += g.sine_gaussian(t[lo:hi], t0, f0, Q, a, ph)
            for key, v in zip(("det", "t0", "f0", "Q", "snr"), (d, t0, f0, Q, s)):
                gl[key].append(v)
    inj = dict(m1=im1, m2=im2, snr=snr, tc=tc, dt_hl=dt_hl, phi=phi, amp=amp)
    return Config2(n2=n2, fs2=fs2, n1=n1, fs1=fs1, f_low=f_low, thr1=3.5, thr2=4.0,
                   window1=int(fs1), window2=int(fs2), shift_s=5.0, n_shifts=n_shifts,
                   coinc_s=0.015, rho_c_thr=7.0, psd1=g.psd_bins(n1, fs1), psd2=g.psd_bins(n2, fs2),
                   coarse_m1=cm1, coarse_m2=cm2, fine_m1=fm1, fine_m2=fm2,
                   nbhd_ptr=ptr, nbhd_idx=idx, nbhd_match=val,
                   strain=strain.astype(np.float32), injections=inj,
                   glitches={k: np.asarray(v) for k, v in gl.items()})


@dataclass
class Config4:
    """Reduced-precision workload: a fine TaylorF2 bank at 4096 Hz on 256 s
    segments (N = 2^20) of two detectors with injections."""
    n: int
    fs: float
    f_low: float
    thr: float
    window: int
    psd: np.ndarray
    m1: np.ndarray
    m2: np.ndarray
    noise_fd: np.ndarray          # complex128 [2, N/2+1]
    inj: dict

    def data_fd(self, device, ld=None):
        """Noise plus injections as a complex64 torch tensor [2, ld] on device
        (the injections are evaluated there with ``taylorf2_torch``)."""
        import torch

        nb = self.n // 2 + 1
        ld = nb if ld is None else ld
        dev = torch.device(device)
        out = torch.zeros((2, ld), dtype=torch.complex128, device=dev)
        out[:, :nb] = torch.from_numpy(self.noise_fd).to(dev)
        f = torch.arange(nb, dtype=torch.float64, device=dev) * (self.fs / self.n)
        w = torch.zeros(nb, dtype=torch.float64, device=dev)
        psd = torch.from_numpy(self.psd).to(dev)
        band = (f >= self.f_low) & (torch.arange(nb, device=dev) < self.n // 2) & (psd > 0)
        w[band] = 4.0 * (self.fs / self.n) / psd[band]
        im1, im2 = self.inj["m1"], self.inj["m2"]
        for b0 in range(0, len(im1), 16):
            b1 = min(len(im1), b0 + 16)
            h = g.taylorf2_torch(self.n, self.fs, im1[b0:b1], im2[b0:b1], self.f_low, dev).to(torch.complex128)
            sig = torch.sqrt((w[None, :] * (h.real ** 2 + h.imag ** 2)).sum(dim=1))
            amp = torch.from_numpy(self.inj["snr"][b0:b1]).to(dev) / sig
            for d in range(2):
                t0 = torch.from_numpy(self.inj["tc"][b0:b1] + (self.inj["dt_hl"][b0:b1] if d == 1 else 0.0)).to(dev)
                ph = torch.from_numpy(self.inj["phi"][b0:b1, d]).to(dev)
                sh = torch.exp(-2j * math.pi * f[None, :] * t0[:, None] + 1j * ph[:, None])
                out[d, :nb] += (amp[:, None] * h * sh).sum(dim=0)
        return out.to(torch.complex64)


def make_config4(seed=4, n_tmpl=50000, n_inj=200, f_low=30.0):
    """50,000 fine templates (chirp mass 1.2-10, the banks' chirp-time
    distribution), 2 detectors x 256 s at 4096 Hz, 200 injections at optimal
    SNR U(5, 30) spread evenly over the segment (dt_HL within 10 ms)."""
    fs, T = 4096.0, 256.0
    n = int(fs * T)
    rng = np.random.default_rng(seed)
    m1, m2, _, _ = g.sample_bank_chirp_times(rng, n_tmpl, f_low)
    noise = np.stack([g.coloured_noise_fd(rng, n, fs) for _ in range(2)])
    im1, im2, _, _ = g.sample_bank_chirp_times(rng, n_inj, f_low)
    slot = T / n_inj
    inj = dict(m1=im1, m2=im2, snr=rng.uniform(5.0, 30.0, n_inj),
               tc=(np.arange(n_inj) + 0.5) * slot + rng.uniform(-0.25, 0.25, n_inj) * slot,
               dt_hl=rng.uniform(-0.010, 0.010, n_inj), phi=rng.uniform(0, 2 * math.pi, (n_inj, 2)))
    return Config4(n=n, fs=fs, f_low=f_low, thr=5.5, window=int(fs), psd=g.psd_bins(n, fs), m1=m1, m2=m2,
                   noise_fd=noise, inj=inj)


@dataclass
class Config3:
    """Uneven-length workload: a TaylorF2 bank with durations of seconds to
    ~100 s, grouped into length classes, over long two-detector data."""
    fs: float
    n_samples: int
    f_low: float
    thr: float
    window: int
    class_len: tuple
    m1: np.ndarray                # per template, ordered by class
    m2: np.ndarray
    duration: np.ndarray          # 2PN duration from f_low, s
    cls: np.ndarray               # length class of each template
    noise_fd: np.ndarray          # complex128 [2, n_fd/2+1] on the grid of n_fd >= n_samples samples
    n_fd: int
    inj: dict

    def class_ids(self, c):
        return np.flatnonzero(self.cls == c)

    def psd(self, n):
        return g.psd_bins(n, self.fs)

    def strain(self, device):
        """float32 torch tensor [2, n_samples] on device: noise plus injections
        (evaluated there with ``taylorf2_torch`` on the n_fd grid)."""
        import torch

        dev = torch.device(device)
        nb = self.n_fd // 2 + 1
        fd = torch.from_numpy(self.noise_fd).to(dev)
        f = torch.arange(nb, dtype=torch.float64, device=dev) * (self.fs / self.n_fd)
        psd = torch.from_numpy(g.psd_bins(self.n_fd, self.fs)).to(dev)
        w = torch.zeros(nb, dtype=torch.float64, device=dev)
        band = (f >= self.f_low) & (torch.arange(nb, device=dev) < self.n_fd // 2) & (psd > 0)
        w[band] = 4.0 * (self.fs / self.n_fd) / psd[band]
        im1, im2 = self.inj["m1"], self.inj["m2"]
        for b0 in range(0, len(im1), 8):
            b1 = min(len(im1), b0 + 8)
            h = g.taylorf2_torch(self.n_fd, self.fs, im1[b0:b1], im2[b0:b1], self.f_low, dev).to(torch.complex128)
            sig = torch.sqrt((w[None, :] * (h.real ** 2 + h.imag ** 2)).sum(dim=1))
            amp = torch.from_numpy(self.inj["snr"][b0:b1]).to(dev) / sig
            for d in range(2):
                t0 = torch.from_numpy(self.inj["tc"][b0:b1] + (self.inj["dt_hl"][b0:b1] if d == 1 else 0.0)).to(dev)
                ph = torch.from_numpy(self.inj["phi"][b0:b1, d]).to(dev)
                sh = torch.exp(-2j * math.pi * f[None, :] * t0[:, None] + 1j * ph[:, None])
                fd[d] += (amp[:, None] * h * sh).sum(dim=0)
            del h
        x = torch.fft.irfft(fd, n=self.n_fd, dim=-1) * self.fs
        return x[:, :self.n_samples].to(torch.float32).contiguous()


def make_config3(seed=3, n_tmpl=20000, T=4096.0, fs=2048.0, f_low=25.0, class_len=(4.0, 16.0, 64.0, 256.0),
                 n_inj=64, margin=1.1):
    """20,000 TaylorF2 templates (chirp mass 1.2-10, durations ~2.5-91 s from
    25 Hz) in 4/16/64/256 s length classes (the smallest class holding
    margin x the 2PN duration), two detectors x 4096 s at 2048 Hz of coloured
    noise with n_inj injections at SNR U(8, 20)."""
    rng = np.random.default_rng(seed)
    m1, m2, _, _ = g.sample_bank_chirp_times(rng, n_tmpl, f_low)
    dur = g.duration_2pn(m1, m2, f_low)
    cls = np.searchsorted(np.asarray(class_len), margin * dur, side="left")
    keep = cls < len(class_len)
    order = np.lexsort((np.arange(n_tmpl)[keep], cls[keep]))
    m1, m2, dur, cls = m1[keep][order], m2[keep][order], dur[keep][order], cls[keep][order]
    n_samples = int(T * fs)
    n_fd = 1 << int(math.ceil(math.log2(n_samples)))
    noise = np.stack([g.coloured_noise_fd(rng, n_fd, fs) for _ in range(2)])
    im1, im2, _, _ = g.sample_bank_chirp_times(rng, n_inj, f_low)
    inj = dict(m1=im1, m2=im2, snr=rng.uniform(8.0, 20.0, n_inj),
               tc=np.sort(rng.uniform(100.0 + 0.1 * T, 0.98 * T, n_inj)), dt_hl=rng.uniform(-0.010, 0.010, n_inj),
               phi=rng.uniform(0, 2 * math.pi, (n_inj, 2)))
    return Config3(fs=fs, n_samples=n_samples, f_low=f_low, thr=5.5, window=int(fs), class_len=tuple(class_len),
                   m1=m1, m2=m2, duration=dur, cls=cls.astype(np.int32), noise_fd=noise, n_fd=n_fd, inj=inj)
