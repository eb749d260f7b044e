"""Learned proposal for the stage-2 follow-up (the workload's learned-ranking
pattern; the paper's own follow-up filters the whole neighbourhood, Sec. III).

The pipeline generates its own training pairs: short segments with one
injected signal each are filtered with the coarse bank at the stage-1 rate;
the loudest coarse trigger is the candidate c*, whose features are the
rho^2-weighted chirp mass and symmetric mass ratio of the coarse triggers
coincident with it, its SNR, its time and the detector; the neighbourhood of
c* is then filtered at the stage-2 rate and the label is the slot of its
loudest fine template.  A network (libmf ``mf_mlp_*`` kernels) learns to rank
the slots; stage 2 can then filter only its top-k slots, with the full
neighbourhood as the fallback.  Every filter and every network step runs in
libmf's CUDA kernels; this module only moves data between them.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import mf

N_FEATURES = 5


@dataclass
class PairSet:
    x: np.ndarray          # float32 [n, 5] raw features (Mc_est, eta_est, snr, t, det)
    n_valid: np.ndarray    # int32 [n] neighbourhood size of c*
    label: np.ndarray      # int32 [n] slot of the loudest fine template
    slot_snr: np.ndarray   # float32 [n, max_slots] stage-2 SNR of every slot (0 if below threshold)
    coarse: np.ndarray     # int32 [n] c*


def generate_pairs(n_pairs, coarse_m1, coarse_m2, fine_m1, fine_m2, nbhd_ptr, nbhd_idx, seed=0, T=32.0,
                   fs1=512.0, fs2=2048.0, f_low=30.0, snr_range=(8.0, 20.0), per_call=64, thr1=5.0, thr2=4.0,
                   max_slots=2000, device="cuda:0"):
    """Training pairs from injection runs filtered by libmf (see the module header)."""
    import torch

    import synth

    dev = torch.device(device)
    rng = np.random.default_rng(seed)
    n1, n2 = int(T * fs1), int(T * fs2)
    nb1, nb2 = n1 // 2 + 1, n2 // 2 + 1
    ld1, ld2 = (nb1 + 63) // 64 * 64, (nb2 + 63) // 64 * 64
    st = torch.cuda.Stream(device=dev)
    p1 = mf.Plan(fs1, n1, per_call, f_low, fs1 / 2, thr1, int(fs1), max_triggers=1 << 22, stream=st.cuda_stream)
    p2 = mf.Plan(fs2, n2, per_call, f_low, fs2 / 2, thr2, int(fs2), max_triggers=1 << 22, stream=st.cuda_stream)
    p1.set_psd(synth.psd_bins(n1, fs1))
    p2.set_psd(synth.psd_bins(n2, fs2))
    p1.bank_reserve(len(coarse_m1))
    for r0, rows in synth.taylorf2_chunks_torch(n1, fs1, coarse_m1, coarse_m2, f_low, dev, chunk=512, ld=ld1):
        p1.bank_set_rows(r0, rows, ld=ld1, on_device=1)
    p2.bank_reserve(len(fine_m1))
    for r0, rows in synth.taylorf2_chunks_torch(n2, fs2, fine_m1, fine_m2, f_low, dev, chunk=256, ld=ld2):
        p2.bank_set_rows(r0, rows, ld=ld2, on_device=1)
    cmc = synth.chirp_mass(coarse_m1, coarse_m2)
    ceta = coarse_m1 * coarse_m2 / (coarse_m1 + coarse_m2) ** 2
    psd2 = torch.from_numpy(synth.psd_bins(n2, fs2)).to(dev)
    f2 = torch.arange(nb2, dtype=torch.float64, device=dev) * (fs2 / n2)
    amp_noise = torch.where((f2 >= 10.0) & (torch.arange(nb2, device=dev) < n2 // 2),
                            torch.sqrt(T * torch.clamp(psd2, min=0) / 4.0), torch.zeros_like(f2))
    d2 = torch.zeros((per_call, ld2), dtype=torch.complex64, device=dev)
    d1 = torch.zeros((per_call, ld1), dtype=torch.complex64, device=dev)
    gen = torch.Generator(device=dev).manual_seed(int(seed))
    xs, nvs, labs, snrs, cs = [], [], [], [], []
    made = 0
    while made < n_pairs:
        # injections: parameters from the bank's distribution, circular in the FD
        im1, im2, _, _ = synth.sample_bank_chirp_times(rng, per_call, f_low)
        snr = rng.uniform(*snr_range, per_call)
        tc = rng.uniform(0.15 * T, 0.85 * T, per_call)
        phi = rng.uniform(0, 2 * math.pi, per_call)
        det = rng.integers(0, 2, per_call)
        h = synth.taylorf2_torch(n2, fs2, im1, im2, f_low, dev, ld=nb2).to(torch.complex128)
        w = torch.zeros(nb2, dtype=torch.float64, device=dev)
        band = (f2 >= f_low) & (torch.arange(nb2, device=dev) < n2 // 2) & (psd2 > 0)
        w[band] = 4.0 * (fs2 / n2) / psd2[band]
        sig = torch.sqrt((w[None, :] * (h.real ** 2 + h.imag ** 2)).sum(dim=1))
        amp = torch.from_numpy(snr).to(dev) / sig
        ph = torch.exp(-2j * math.pi * f2[None, :] * torch.from_numpy(tc).to(dev)[:, None]
                       + 1j * torch.from_numpy(phi).to(dev)[:, None])
        a = torch.randn((per_call, nb2), dtype=torch.float64, device=dev, generator=gen)
        b = torch.randn((per_call, nb2), dtype=torch.float64, device=dev, generator=gen)
        fd = amp_noise[None, :] * torch.complex(a, b) + amp[:, None] * h * ph
        d2[:, :nb2] = fd.to(torch.complex64)
        torch.cuda.current_stream(dev).synchronize()
        p1.decimate(d2, d1, ld_in=ld2, ld_out=ld1)
        p1.filter(d1, ld=ld1)
        t1, _, _ = p1.triggers()
        cand = []
        for d in range(per_call):
            td = t1[t1["det"] == d]
            if len(td) == 0:
                cand.append(None)
                continue
            i = int(np.argmax(td["snr"]))
            c, s1, r1 = int(td["tmpl"][i]), int(td["sample"][i]), float(td["snr"][i])
            near = td[np.abs(td["sample"] - s1) <= int(0.015 * fs1)]
            wgt = near["snr"].astype(np.float64) ** 2
            mc_est = float((wgt * cmc[near["tmpl"]]).sum() / wgt.sum())
            eta_est = float((wgt * ceta[near["tmpl"]]).sum() / wgt.sum())
            lo, hi = int(nbhd_ptr[c]), int(nbhd_ptr[c + 1])
            if hi == lo:
                cand.append(None)
                continue
            cand.append((c, s1, r1, mc_est, eta_est, np.asarray(nbhd_idx[lo:hi])))
        union = np.unique(np.concatenate([cd[5] for cd in cand if cd is not None] or [np.zeros(0, np.int32)]))
        if len(union) == 0:
            continue
        sub = torch.from_numpy(union.astype(np.int32)).to(dev)
        p2.filter(d2, subset=sub, ld=ld2)
        t2, _, _ = p2.triggers()
        for d, cd in enumerate(cand):
            if cd is None or made >= n_pairs:
                continue
            c, s1, r1, mc_est, eta_est, nb = cd
            td = t2[(t2["det"] == d) & (np.abs(t2["sample"] - 4 * s1) <= int(0.03 * fs2))]
            slot_snr = np.zeros(max_slots, np.float32)
            best = {}
            for tr in td:
                best[int(tr["tmpl"])] = max(best.get(int(tr["tmpl"]), 0.0), float(tr["snr"]))
            vals = np.array([best.get(int(f), 0.0) for f in nb], np.float32)
            if vals.max() <= 0:
                continue
            slot_snr[:len(nb)] = vals
            xs.append([mc_est, eta_est, r1, s1 / fs1, float(det[d])])
            nvs.append(len(nb))
            labs.append(int(np.argmax(vals)))
            snrs.append(slot_snr)
            cs.append(c)
            made += 1
    p1.close()
    p2.close()
    return PairSet(np.array(xs, np.float32), np.array(nvs, np.int32), np.array(labs, np.int32),
                   np.stack(snrs), np.array(cs, np.int32))


class Proposal:
    """The trained ranking network with its feature normalisation."""

    def __init__(self, width=256, depth=4, n_out=2000, max_batch=1024, device="cuda:0"):
        import torch

        self.torch = torch
        self.dev = torch.device(device)
        self.net = mf.MLP(N_FEATURES, width, depth, n_out, max_batch)
        self.n_out, self.max_batch = n_out, max_batch
        self.mu = np.zeros(N_FEATURES, np.float32)
        self.sd = np.ones(N_FEATURES, np.float32)

    def norm(self, x):
        return ((x - self.mu) / self.sd).astype(np.float32)

    def init(self, seed=0):
        from math import sqrt
        rng = np.random.default_rng(seed)
        n_in, w, depth, n_out = N_FEATURES, self.net.dims[1], self.net.dims[2], self.net.dims[3]
        parts, d = [], n_in
        for li in range(depth + 1):
            o = w if li < depth else n_out
            parts.append(rng.standard_normal(d * o) * sqrt(2.0 / d))
            parts.append(np.zeros(o))
            d = w
        self.net.set_params(np.concatenate(parts).astype(np.float32))

    def fit(self, pairs: PairSet, epochs=30, lr=2e-3, batch=1024, seed=0, weight_decay=1e-4):
        torch = self.torch
        self.mu = pairs.x.mean(axis=0)
        self.sd = pairs.x.std(axis=0) + 1e-6
        x = torch.from_numpy(self.norm(pairs.x)).to(self.dev)
        nv = torch.from_numpy(pairs.n_valid).to(self.dev)
        lab = torch.from_numpy(pairs.label).to(self.dev)
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        rng = np.random.default_rng(seed)
        n = len(pairs.x)
        hist = []
        for ep in range(epochs):
            perm = torch.from_numpy(rng.permutation(n)).to(self.dev)
            tot = 0.0
            nb = 0
            for b0 in range(0, n - batch + 1, batch):
                idx = perm[b0:b0 + batch]
                xb, nvb, lb = x[idx].contiguous(), nv[idx].contiguous(), lab[idx].contiguous()
                self.net.loss_grad(xb, nvb, lb, loss=loss)
                self.net.adamw_step(lr * 0.5 * (1 + math.cos(math.pi * ep / epochs)), weight_decay=weight_decay)
                tot += float(loss.item())
                nb += 1
            hist.append(tot / max(nb, 1))
        return hist

    def rank(self, x, n_valid, k, p_mass=2.0):
        """Proposed slots (int32 [n, k], -1 padded) for raw features x: the top
        k, or fewer once their probability reaches p_mass."""
        torch = self.torch
        out = []
        for b0 in range(0, len(x), self.max_batch):
            xb = torch.from_numpy(self.norm(x[b0:b0 + self.max_batch])).to(self.dev)
            nvb = torch.from_numpy(np.ascontiguousarray(n_valid[b0:b0 + self.max_batch])).to(self.dev)
            o = torch.zeros((len(xb), k), dtype=torch.int32, device=self.dev)
            self.net.topk(xb, nvb, k, o, p_mass=p_mass)
            out.append(o.cpu().numpy())
        return np.concatenate(out)


def recovered(slot_snr, n_valid, chosen):
    """Best SNR among the chosen slots / best SNR in the whole neighbourhood, and
    the number of templates filtered (chosen slots, capped at the neighbourhood)."""
    best = np.array([slot_snr[i, :n_valid[i]].max() for i in range(len(n_valid))])
    got = np.array([max([slot_snr[i, j] for j in chosen[i] if j >= 0] or [0.0]) for i in range(len(n_valid))])
    used = np.array([min(int((chosen[i] >= 0).sum()), int(n_valid[i])) for i in range(len(n_valid))])
    return got / best, used
