"""Exact-match neighbourhoods of the coarse bank in the fine bank (Sec. III:
stage 2 filters the templates "in the vicinity" of a followed coarse
template; the workload fixes the vicinity as match >= 0.9).

match(c, f) = max over t_c and phase of (h_c, h_f(t_c)) / (sigma_c sigma_f)
(Eq. 2 inner product) is computed with the filter itself: the coarse template
scaled by 1 / sigma_c is the data, the fine templates are the bank, and with a
single clustering window spanning the whole (circular) segment every trigger
is (coarse row, fine template, max over t_c of rho) = the match.  A cheaper
candidate list (e.g. the quadratic-metric map at a looser threshold) limits
the fine templates filtered for each block of coarse templates; every
template of the candidate union is filtered against every coarse row of the
block, and every pair with match >= min_match is kept.  Templates are
generated on the GPU (mf_taylorf2) and every filter step runs in libmf's
kernels; this module only moves data between them.  An untimed set-up step.
"""

from __future__ import annotations

import numpy as np

from . import mf


def exact_nbhd(c_m1, c_m2, f_m1, f_m2, f_low, fs, n, min_match=0.9, cand_ptr=None, cand_idx=None, rows=16,
               max_size=2000, device="cuda:0"):
    """CSR map coarse -> fine of every pair with match >= min_match, slots in
    decreasing match (ties: lower fine id), at most max_size per coarse
    template.  Returns (ptr int64 [n_c + 1], idx int32, match float64).
    cand_ptr / cand_idx: optional candidate CSR (a superset of each
    neighbourhood); None filters every fine template."""
    import torch

    import synth

    dev = torch.device(device)
    c_m1 = np.asarray(c_m1, dtype=np.float64)
    c_m2 = np.asarray(c_m2, dtype=np.float64)
    nc, nf = len(c_m1), len(f_m1)
    nb = n // 2 + 1
    ld = (nb + 63) // 64 * 64
    psd = synth.psd_bins(n, fs)
    lib = mf.load()
    st = torch.cuda.Stream(device=dev)
    # sigma_c of the coarse templates (the library's float64 norms), from a plan holding them as its bank
    pc = mf.Plan(fs, n, 1, f_low, fs / 2, 1.0, n, stream=st.cuda_stream)
    pc.set_psd(psd)
    pc.bank_reserve(nc)
    pc.bank_generate_taylorf2(0, c_m1, c_m2, f_low)
    sig_c = np.sqrt(pc.sigmasq(nc))
    pc.close()
    # the fine bank and a plan whose data rows are `rows` scaled coarse templates, one window of n samples
    p = mf.Plan(fs, n, rows, f_low, fs / 2, min_match, n, max_triggers=1 << 24, stream=st.cuda_stream)
    p.set_psd(psd)
    p.bank_reserve(nf)
    p.bank_generate_taylorf2(0, f_m1, f_m2, f_low)
    with torch.cuda.stream(st):  # every torch op on the plans' stream
        data = torch.zeros((rows, ld), dtype=torch.complex64, device=dev)
        cs_l, fi_l, ms_l = [], [], []
        for c0 in range(0, nc, rows):
            c1 = min(nc, c0 + rows)
            data.zero_()
            a1 = np.ascontiguousarray(c_m1[c0:c1])
            a2 = np.ascontiguousarray(c_m2[c0:c1])
            rc = lib.mf_taylorf2(a1.ctypes.data, a2.ctypes.data, c1 - c0, fs, n, f_low, mf._ptr(data), ld,
                                 st.cuda_stream)
            if rc != mf.MF_OK:
                raise mf.MFError(rc, lib.mf_last_error(None).decode())
            data[: c1 - c0] /= torch.from_numpy(sig_c[c0:c1]).to(dev, torch.float32)[:, None]
            if cand_ptr is None:
                sub = None
            else:
                parts = [np.asarray(cand_idx[cand_ptr[c]:cand_ptr[c + 1]]) for c in range(c0, c1)]
                u = np.unique(np.concatenate(parts)) if parts else np.zeros(0, np.int32)
                if len(u) == 0:
                    continue
                sub = torch.from_numpy(u.astype(np.int32)).to(dev)
            p.filter(data, subset=sub, ld=ld)
            trig, _, _ = p.triggers()
            keep = trig["det"] < c1 - c0
            cs_l.append(trig["det"][keep].astype(np.int64) + c0)
            fi_l.append(trig["tmpl"][keep].astype(np.int64))
            ms_l.append(trig["snr"][keep].astype(np.float64))
    p.close()
    cs = np.concatenate(cs_l) if cs_l else np.zeros(0, np.int64)
    fs_ = np.concatenate(fi_l) if fi_l else np.zeros(0, np.int64)
    ms = np.concatenate(ms_l) if ms_l else np.zeros(0)
    order = np.lexsort((fs_, -ms, cs))  # by coarse, then decreasing match, then fine id
    cs, fs_, ms = cs[order], fs_[order], ms[order]
    ptr = np.zeros(nc + 1, dtype=np.int64)
    idx_l, val_l = [], []
    for c in range(nc):
        lo, hi = np.searchsorted(cs, [c, c + 1])
        take = slice(lo, min(hi, lo + max_size))
        idx_l.append(fs_[take].astype(np.int32))
        val_l.append(ms[take])
        ptr[c + 1] = ptr[c] + len(idx_l[-1])
    return ptr, np.concatenate(idx_l), np.concatenate(val_l)


def exact_nbhd_of_config(coarse_m1, coarse_m2, fine_m1, fine_m2, f_low=30.0, fs=2048.0, n=1 << 18,
                         min_match=0.9, cand_match=0.8, device="cuda:0"):
    """Exact neighbourhoods of a coarse / fine bank pair at the stage-2 rate:
    candidates from the quadratic-metric map at cand_match (the metric agrees
    with the exact match to a few 1e-2 on the workload's banks, so the
    candidates hold every member), the match over a segment longer than every
    template (2^18 samples at 2048 Hz, 128 s).  Returns (ptr, idx, match)."""
    import synth

    cptr, cidx, _ = synth.nbhd_map(coarse_m1, coarse_m2, fine_m1, fine_m2, f_low, f_low, fs / 2,
                                   min_match=cand_match)
    return exact_nbhd(coarse_m1, coarse_m2, fine_m1, fine_m2, f_low, fs, n, min_match=min_match, cand_ptr=cptr,
                      cand_idx=cidx, device=device)
