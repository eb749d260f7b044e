"""GPU parity of the FP16-intermediate filter with the tensor-core row pass
(mf_set_intermediate(MF_F16), N = 2^20) against the FP64 oracle: every window
peak of every template in coloured noise with a loud glitch and a TaylorF2
injection, SNR within 1e-3 relative (the workload's SNR-error bar) with the
near-tie allowances scaled to that bar; the injected template's peak at its
sample with rho = A sigma; several launches per call, subsets, one and two
detectors; agreement with the FP32 path; and the argument checks.  The same
for the FP16-pair intermediate with split tensor-core products
(mf_set_intermediate(MF_F16X2)) at the FP32 path's bar, 1e-4."""

import math

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O
from tests.parity import compare_triggers, oracle_rho2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
N, FS, F_LOW = 1 << 20, 2048.0, 30.0
SNR_RTOL, REL_TIE = 1e-3, 2e-3  # rho to 1e-3, so rho^2 ties and threshold edges to 2e-3
SPLIT_RTOL, SPLIT_TIE = 1e-4, 2e-4  # FP16 pairs: the FP32 bar


@pytest.fixture(scope="module")
def case(lib):
    rng = np.random.default_rng(20)
    n_tmpl = 12
    m1, m2 = synth.sample_bank_uniform_masses(rng, n_tmpl, 1.4, 10.0)
    psd = synth.psd_bins(N, FS)
    w = O.weights(N, FS, F_LOW, FS / 2, psd)
    bank = synth.taylorf2_torch(N, FS, m1, m2, F_LOW, DEV)
    bank_np = bank.cpu().numpy()
    fd = np.stack([synth.coloured_noise_fd(rng, N, FS) for _ in range(2)])
    inj, t_inj, snr_inj = 7, 200.0, 12.0
    sig = math.sqrt(O.sigmasq(bank_np[inj].astype(np.complex128), w))
    amp = snr_inj / sig
    # injection built from the stored template itself: a circular shift to sample j0 in the FD
    j0 = int(t_inj * FS)
    k = np.arange(N // 2 + 1)
    fd[1] += amp * bank_np[inj].astype(np.complex128) * np.exp(-2j * np.pi * k * j0 / N)
    t = np.arange(N) / FS
    a = synth.sine_gaussian_amplitude(400.0, 150.0, 6.0)
    fd[0] += O.strain_to_fd(synth.sine_gaussian(t, 300.0, 150.0, 6.0, a, 0.3), FS)
    fd = fd.astype(np.complex64)
    rho2, z = oracle_rho2(fd.astype(np.complex128), bank_np.astype(np.complex128), psd, N, FS, F_LOW, FS / 2)
    return dict(psd=psd, bank=bank, bank_np=bank_np, fd=fd, rho2=rho2, z=z, inj=inj, j0=j0, snr_inj=snr_inj)


def _filter(mf, c, n_det=2, inter=None, batch=None, subset=None, thr=4.0):
    p = mf.Plan(FS, N, n_det, F_LOW, FS / 2, thr, int(FS), max_triggers=1 << 20)
    p.set_psd(c["psd"])
    p.load_bank(c["bank"])
    if inter is not None:
        p.set_intermediate(inter)
    if batch is not None:
        p.set_batch(batch)
    d = torch.from_numpy(c["fd"][2 - n_det:]).to(DEV)
    if subset is None:
        p.filter(d)
    else:
        p.filter(d, subset=torch.tensor(subset, dtype=torch.int32, device=DEV), n_subset=len(subset))
    trig, n, _ = p.triggers()
    st = p.stats()
    p.close()
    return trig, n, st


def test_tc_row_pass_matches_the_oracle(case):
    from paper_2309_00019_gb300 import mf

    trig, n, st = _filter(mf, case, inter=mf.MF_F16)
    assert st["impl"] == 3 and n == len(trig) > 0
    ids = list(range(len(case["bank_np"])))
    res = compare_triggers(trig, case["rho2"], ids, 4.0, int(FS), rel_tie=REL_TIE, snr_rtol=SNR_RTOL,
                           phase_atol=0.01, z=case["z"])
    assert res["exact"] > 0.99 * n
    # the injection: its window peak at the injected sample (rho = A sigma plus a unit complex Gaussian)
    i = np.nonzero((trig["det"] == 1) & (trig["tmpl"] == case["inj"]) & (trig["sample"] == case["j0"]))[0]
    assert len(i) == 1 and abs(trig["snr"][i[0]] - case["snr_inj"]) < 4.0
    # the glitch (rho ~ 400 in the loudest templates) is inside FP16's range
    assert trig["snr"][trig["det"] == 0].max() > 100
    print(f"\nFP16 intermediate + tensor-core rows: {n} triggers, {res}")


def test_tc_row_pass_noiseless_injection_recovers_a_sigma(case):
    from paper_2309_00019_gb300 import mf

    # data = the injection alone (no noise): rho at the injected sample is exactly A sigma = 12 (Eq. 2)
    bank_np, inj, j0 = case["bank_np"], case["inj"], case["j0"]
    w = O.weights(N, FS, F_LOW, FS / 2, case["psd"])
    amp = case["snr_inj"] / math.sqrt(O.sigmasq(bank_np[inj].astype(np.complex128), w))
    k = np.arange(N // 2 + 1)
    d = (amp * bank_np[inj].astype(np.complex128) * np.exp(-2j * np.pi * k * j0 / N))[None].astype(np.complex64)
    c = dict(case, fd=np.concatenate([d, d]))
    trig, n, st = _filter(mf, c, n_det=1, inter=mf.MF_F16, subset=[inj], thr=6.0)
    assert st["impl"] == 3
    i = np.nonzero(trig["sample"] == j0)[0]
    assert len(i) == 1 and abs(trig["snr"][i[0]] / case["snr_inj"] - 1) < 1e-3, trig
    print(f"\nnoiseless injection: rho {trig['snr'][i[0]]:.6f} (A sigma = {case['snr_inj']})")


def test_tc_row_pass_batches_subsets_one_detector(case):
    from paper_2309_00019_gb300 import mf

    sub = [11, 3, 7, 0, 5]
    trig, n, st = _filter(mf, case, n_det=1, inter=mf.MF_F16, batch=2, subset=sub)
    assert st["impl"] == 3
    assert set(np.unique(trig["tmpl"]).tolist()) <= set(sub) and n > 0
    rho2 = case["rho2"][1:, sub]
    res = compare_triggers(trig, rho2, sub, 4.0, int(FS), rel_tie=REL_TIE, snr_rtol=SNR_RTOL)
    assert res["exact"] > 0.99 * n


def test_tc_row_pass_agrees_with_the_fp32_path(case):
    from paper_2309_00019_gb300 import mf

    a, na, sa = _filter(mf, case, inter=mf.MF_F16)
    b, nb, sb = _filter(mf, case)
    assert sa["impl"] == 3 and sb["impl"] == 2
    ka = {(int(t["det"]), int(t["tmpl"]), int(t["sample"])): float(t["snr"]) for t in a}
    kb = {(int(t["det"]), int(t["tmpl"]), int(t["sample"])): float(t["snr"]) for t in b}
    common = ka.keys() & kb.keys()
    assert len(common) >= 0.99 * max(len(ka), len(kb))
    worst = max(abs(ka[k] - kb[k]) / kb[k] for k in common)
    assert worst <= SNR_RTOL
    print(f"\nFP16 + tensor cores vs FP32 path: {len(common)} common window peaks of {len(kb)}, "
          f"max rel SNR diff {worst:.2e}")


def test_split_row_pass_matches_the_oracle_at_the_fp32_bar(case):
    from paper_2309_00019_gb300 import mf

    trig, n, st = _filter(mf, case, inter=mf.MF_F16X2)
    assert st["impl"] == 4 and n == len(trig) > 0
    ids = list(range(len(case["bank_np"])))
    res = compare_triggers(trig, case["rho2"], ids, 4.0, int(FS), rel_tie=SPLIT_TIE, snr_rtol=SPLIT_RTOL,
                           phase_atol=0.01, z=case["z"])
    assert res["exact"] > 0.99 * n
    i = np.nonzero((trig["det"] == 1) & (trig["tmpl"] == case["inj"]) & (trig["sample"] == case["j0"]))[0]
    assert len(i) == 1
    assert trig["snr"][trig["det"] == 0].max() > 100
    print(f"\nFP16-pair intermediate + split tensor-core products: {n} triggers, {res}")


def test_split_row_pass_noiseless_injection_and_batches(case):
    from paper_2309_00019_gb300 import mf

    bank_np, inj, j0 = case["bank_np"], case["inj"], case["j0"]
    w = O.weights(N, FS, F_LOW, FS / 2, case["psd"])
    amp = case["snr_inj"] / math.sqrt(O.sigmasq(bank_np[inj].astype(np.complex128), w))
    k = np.arange(N // 2 + 1)
    d = (amp * bank_np[inj].astype(np.complex128) * np.exp(-2j * np.pi * k * j0 / N))[None].astype(np.complex64)
    c = dict(case, fd=np.concatenate([d, d]))
    trig, n, st = _filter(mf, c, n_det=1, inter=mf.MF_F16X2, subset=[inj], thr=6.0)
    i = np.nonzero(trig["sample"] == j0)[0]
    assert st["impl"] == 4 and len(i) == 1 and abs(trig["snr"][i[0]] / case["snr_inj"] - 1) < 1e-5, trig
    sub = [11, 3, 7, 0, 5]
    trig, n, st = _filter(mf, case, n_det=1, inter=mf.MF_F16X2, batch=2, subset=sub)
    res = compare_triggers(trig, case["rho2"][1:, sub], sub, 4.0, int(FS), rel_tie=SPLIT_TIE, snr_rtol=SPLIT_RTOL)
    assert n > 0 and res["exact"] > 0.99 * n


def test_split_row_pass_agrees_with_the_fp32_path(case):
    from paper_2309_00019_gb300 import mf

    a, na, sa = _filter(mf, case, inter=mf.MF_F16X2)
    b, nb, sb = _filter(mf, case)
    assert sa["impl"] == 4 and sb["impl"] == 2
    ka = {(int(t["det"]), int(t["tmpl"]), int(t["sample"])): float(t["snr"]) for t in a}
    kb = {(int(t["det"]), int(t["tmpl"]), int(t["sample"])): float(t["snr"]) for t in b}
    common = ka.keys() & kb.keys()
    assert len(common) >= 0.999 * max(len(ka), len(kb))
    worst = max(abs(ka[k] - kb[k]) / kb[k] for k in common)
    assert worst <= SPLIT_RTOL
    print(f"\nFP16 pairs + split products vs FP32 path: {len(common)} common window peaks of {len(kb)}, "
          f"max rel SNR diff {worst:.2e}")


def test_set_intermediate_argument_checks(lib):
    from paper_2309_00019_gb300 import mf

    p = mf.Plan(512.0, 1 << 14, 1, 30.0, 256.0, 5.0, 512)
    with pytest.raises(mf.MFError):
        p.set_intermediate(mf.MF_F16)  # N != 2^20
    with pytest.raises(mf.MFError):
        p.set_intermediate(mf.MF_F16X2)
    p.set_intermediate(mf.MF_F32)
    with pytest.raises(mf.MFError):
        p.set_intermediate(mf.MF_BF16)
    p.close()


def test_tc_empty_subset_and_small_trigger_buffer(case):
    """Both FP16 intermediates: a call that selects no template gives no trigger, and a trigger buffer smaller
    than the count returns its first records with the full count and MF_EOVERFLOW."""
    from paper_2309_00019_gb300 import mf

    d = torch.from_numpy(case["fd"]).to(DEV)
    for inter in (mf.MF_F16, mf.MF_F16X2):
        p = mf.Plan(FS, N, 2, F_LOW, FS / 2, 4.0, int(FS), max_triggers=1 << 20)
        p.set_psd(case["psd"])
        p.load_bank(case["bank"])
        p.set_intermediate(inter)
        p.filter(d, subset=torch.zeros(0, dtype=torch.int32, device=DEV), n_subset=0)
        trig, n0, _ = p.triggers()
        assert n0 == 0 and len(trig) == 0
        p.filter(d)
        full, n_all, _ = p.triggers()
        part, n_part, st = p.triggers(cap=5)
        assert n_all > 5 and n_part == n_all and len(part) == 5 and st == mf.MF_EOVERFLOW
        assert np.array_equal(part, full[:5])
        p.close()


def test_profiling_times_every_kth_launch_pair(case):
    """mf_profile(k): the CUDA-event counters cover every k-th launch pair (counted across calls); profiling
    changes no trigger."""
    from paper_2309_00019_gb300 import mf

    d = torch.from_numpy(case["fd"]).to(DEV)
    p = mf.Plan(FS, N, 2, F_LOW, FS / 2, 4.0, int(FS), max_triggers=1 << 20)
    p.set_psd(case["psd"])
    p.load_bank(case["bank"])
    p.set_intermediate(mf.MF_F16)
    p.set_batch(1)  # 12 templates: 12 launch pairs per call
    p.filter(d)
    ref = p.triggers()[0].copy()
    for k, want in ((1, 24), (2, 12), (5, 5)):
        p.stats(reset=True)
        p.profile(k)
        p.filter(d)
        p.filter(d)
        st = p.stats(reset=True)
        assert st["pass1_launches"] == st["pass2_launches"] == want, (k, st)
        assert st["pass1_series"] == 2 * want and st["pass1_ms"] > 0 and st["pass2_ms"] > 0
        assert np.array_equal(p.triggers()[0], ref)
    p.profile(0)
    with pytest.raises(mf.MFError):
        p.profile(-1)
    p.close()
