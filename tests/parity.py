"""Helpers that compare the CUDA path's triggers with the FP64 oracle.

A trigger set is bit-exact in (det, tmpl, sample) apart from documented
near-ties:
  (i)  two samples of one window whose oracle rho^2 differ by <= rel_tie * rho^2
       may swap as the window peak;
  (ii) a window whose oracle peak satisfies |rho^2 - thr^2| <= rel_tie * thr^2
       may be present or absent.
SNR of every matched trigger must agree to ``snr_rtol`` relative.
"""

from __future__ import annotations

import numpy as np

from oracle import mf_oracle as O


def oracle_rho2(stilde, bank_rows, psd, n, fs, f_low, f_high):
    """Full oracle rho^2 series [n_det, n_tmpl, N] and z for rows of a bank."""
    w = O.weights(n, fs, f_low, f_high, psd)
    stilde = np.atleast_2d(stilde)
    out = np.zeros((stilde.shape[0], len(bank_rows), n))
    zz = np.zeros((stilde.shape[0], len(bank_rows), n), dtype=np.complex128)
    for d in range(stilde.shape[0]):
        for i, h in enumerate(bank_rows):
            r2, z = O.snr_squared(stilde[d], np.asarray(h, dtype=np.complex128), w, n)
            out[d, i] = r2
            zz[d, i] = z
    return out, zz


def compare_triggers(gpu, rho2, tmpl_ids, thr, window, valid_begin=0, valid_end=None, rel_tie=1e-4,
                     snr_rtol=1e-4, phase_atol=None, z=None):
    """Check GPU triggers against oracle rho^2 series.

    gpu: structured array with det, tmpl, sample, snr (phase optional).
    rho2: [n_det, len(tmpl_ids), N] oracle series for those templates.
    Returns a dict of statistics; raises AssertionError on a violation.
    """
    n_det, _, n = rho2.shape
    valid_end = n if valid_end is None else valid_end
    thr2 = thr * thr
    pos = {int(t): i for i, t in enumerate(tmpl_ids)}
    got = {}
    for g in gpu:
        key = (int(g["det"]), int(g["tmpl"]), int(g["sample"]) // window)
        assert key not in got, f"two triggers in one window: {key}"
        got[key] = g
    n_exact = n_tie_swap = n_edge = 0
    max_rel = 0.0
    w_first = valid_begin // window
    w_last = (valid_end - 1) // window
    for d in range(n_det):
        for t, i in pos.items():
            r = rho2[d, i]
            for wi in range(w_first, w_last + 1):
                a = max(wi * window, valid_begin)
                b = min((wi + 1) * window, valid_end)
                seg = r[a:b]
                j = int(np.argmax(seg))
                peak = seg[j]
                g = got.pop((d, t, wi), None)
                if peak >= thr2:
                    if g is None:
                        assert peak <= thr2 * (1 + rel_tie), f"missing trigger d={d} t={t} w={wi} rho2={peak}"
                        n_edge += 1
                        continue
                else:
                    if g is not None:
                        assert peak >= thr2 * (1 - rel_tie), \
                            f"extra trigger d={d} t={t} w={wi} rho2={peak} gpu={g}"
                        n_edge += 1
                        continue
                    continue
                s = int(g["sample"])
                assert a <= s < b, f"trigger outside window/valid range: {g}"
                if s == a + j:
                    n_exact += 1
                else:
                    assert r[s] >= peak * (1 - rel_tie), f"wrong peak d={d} t={t} w={wi}: gpu {s} {r[s]} vs {a+j} {peak}"
                    n_tie_swap += 1
                rel = abs(float(g["snr"]) - np.sqrt(r[s])) / np.sqrt(r[s])
                max_rel = max(max_rel, rel)
                assert rel <= snr_rtol, f"snr mismatch d={d} t={t} s={s}: gpu {g['snr']} oracle {np.sqrt(r[s])}"
                if phase_atol is not None and z is not None:
                    ph = np.angle(z[d, i, s])
                    dphi = abs((float(g["phase"]) - ph + np.pi) % (2 * np.pi) - np.pi)
                    assert dphi <= phase_atol, f"phase mismatch {g['phase']} vs {ph}"
    assert not got, f"triggers for templates/windows not expected: {list(got)[:5]}"
    return dict(exact=n_exact, tie_swaps=n_tie_swap, edge=n_edge, max_rel_snr=max_rel)


def _coincide_group(args):
    trig, ring_begin, ring_end, shift_samples, n_shifts, window_samples, rho_c_thr = args
    return O.coincide(trig, ring_begin, ring_end, shift_samples, n_shifts, window_samples, rho_c_thr=rho_c_thr)


def coincide_all_cores(trig, ring_begin, ring_end, shift_samples, n_shifts, window_samples, rho_c_thr,
                       n_workers=None):
    """The oracle's coincide over a large trigger list, split by template across
    a spawn-started process pool (coincidences never pair two templates, so the
    split is exact); result sorted as coincide sorts it."""
    import multiprocessing as mp
    import os

    tm = np.unique(trig["tmpl"])
    n_workers = max(1, min(n_workers or os.cpu_count() or 1, len(tm)))
    groups = [trig[np.isin(trig["tmpl"], g)] for g in np.array_split(tm, 4 * n_workers) if len(g)]
    jobs = [(g, ring_begin, ring_end, shift_samples, n_shifts, window_samples, rho_c_thr) for g in groups]
    with mp.get_context("spawn").Pool(n_workers) as pool:
        parts = pool.map(_coincide_group, jobs)
    parts = [p for p in parts if len(p)]
    out = np.concatenate(parts) if parts else np.zeros(0, O.COINC_DTYPE)
    return np.sort(out, order=["tmpl", "shift", "sample0", "sample1"])
