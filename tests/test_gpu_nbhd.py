"""Exact-match neighbourhoods (Sec. III: the fine templates in the vicinity
of a coarse template; match >= 0.9) computed with the filter itself
(nbhd.exact_nbhd), against the FP64 oracle's match of every pair for a
sample of coarse templates, with candidates from the quadratic-metric map
giving the same result as filtering every fine template, and the metric map
checked against it."""

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FS, N, F_LOW = 2048.0, 1 << 16, 30.0  # 32 s segments, as the learned proposal's runs


@pytest.fixture(scope="module")
def banks(lib):
    # a narrow chirp-mass range, so that 600 fine templates give neighbourhoods of tens of slots
    rng = np.random.default_rng(8)
    cm1, cm2, _, _ = synth.sample_bank_chirp_times(rng, 40, F_LOW, mc_lo=1.2, mc_hi=1.5)
    fm1, fm2, _, _ = synth.sample_bank_chirp_times(rng, 600, F_LOW, mc_lo=1.2, mc_hi=1.5)
    return cm1, cm2, fm1, fm2


def test_exact_neighbourhoods_match_the_oracle(banks):
    from paper_2309_00019_gb300.nbhd import exact_nbhd

    cm1, cm2, fm1, fm2 = banks
    ptr, idx, val = exact_nbhd(cm1, cm2, fm1, fm2, F_LOW, FS, N)
    assert ptr[-1] == len(idx) > 0
    psd = synth.psd_bins(N, FS)
    w = O.weights(N, FS, F_LOW, FS / 2, psd)
    worst, n_pairs = 0.0, 0
    for c in (0, 13, 27, 39):  # every fine template against four coarse templates
        hc = synth.taylorf2(N, FS, cm1[c], cm2[c], F_LOW)
        m = np.array([O.match(hc, synth.taylorf2(N, FS, fm1[f], fm2[f], F_LOW), w, N) for f in range(len(fm1))])
        got = dict(zip(idx[ptr[c]:ptr[c + 1]].tolist(), val[ptr[c]:ptr[c + 1]].tolist()))
        want = set(np.nonzero(m >= 0.9)[0].tolist())
        for f in set(got) ^ want:  # membership differs only at the threshold
            assert abs(m[f] - 0.9) <= 1e-5, (c, f, m[f])
        for f in set(got) & want:
            worst = max(worst, abs(got[f] - m[f]))
            n_pairs += 1
        # slots in decreasing match, ties to the lower id
        vv = val[ptr[c]:ptr[c + 1]]
        assert np.all(np.diff(vv) <= 0)
    # the match value of every member of every neighbourhood
    for c in range(len(cm1)):
        hc = synth.taylorf2(N, FS, cm1[c], cm2[c], F_LOW)
        for f, v in zip(idx[ptr[c]:ptr[c + 1]], val[ptr[c]:ptr[c + 1]]):
            worst = max(worst, abs(v - O.match(hc, synth.taylorf2(N, FS, fm1[f], fm2[f], F_LOW), w, N)))
            n_pairs += 1
    assert n_pairs >= 20 and worst <= 1e-5
    print(f"\nexact neighbourhoods: {len(idx)} pairs, mean size {len(idx) / len(cm1):.1f}; "
          f"{n_pairs} pairs against the oracle's match, max |diff| {worst:.2e}")


def test_metric_candidates_give_the_same_neighbourhoods(banks):
    from paper_2309_00019_gb300.nbhd import exact_nbhd

    cm1, cm2, fm1, fm2 = banks
    full = exact_nbhd(cm1, cm2, fm1, fm2, F_LOW, FS, N)
    cptr, cidx, _ = synth.nbhd_map(cm1, cm2, fm1, fm2, F_LOW, F_LOW, FS / 2, min_match=0.8)
    cand = exact_nbhd(cm1, cm2, fm1, fm2, F_LOW, FS, N, cand_ptr=cptr, cand_idx=cidx)
    assert np.array_equal(full[0], cand[0]) and np.array_equal(full[1], cand[1])
    # the metric map at 0.9 against the exact one: its match values within 0.04 for shared members (the
    # candidate list at 0.8 is then a superset of every exact neighbourhood)
    mptr, midx, mval = synth.nbhd_map(cm1, cm2, fm1, fm2, F_LOW, F_LOW, FS / 2, min_match=0.9)
    ptr, idx, val = full
    shared = tot = 0
    for c in range(len(cm1)):
        e = dict(zip(idx[ptr[c]:ptr[c + 1]].tolist(), val[ptr[c]:ptr[c + 1]].tolist()))
        mm = dict(zip(midx[mptr[c]:mptr[c + 1]].tolist(), mval[mptr[c]:mptr[c + 1]].tolist()))
        tot += len(e)
        for f in e.keys() & mm.keys():
            shared += 1
            assert abs(e[f] - mm[f]) <= 0.04
    print(f"\nmetric map at 0.9 holds {shared} of the {tot} exact members")
    assert shared >= 0.5 * tot
