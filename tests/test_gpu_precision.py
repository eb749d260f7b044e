"""GPU checks of reduced-precision storage: the device quantiser against the
oracle's rounding rule, and the SNR error and trigger-set differences of FP16
and bfloat16 banks and data against the FP64 oracle (exact, unquantised
inputs) and against the FP32 CUDA path.

Tolerances come from the error model pinned in tests/test_quant_oracle_pins.py:
each quantised operand perturbs rho by an additive error of standard deviation
about 0.45 u (u = 2^-11 for FP16, 2^-8 for bfloat16), so bank plus data give
sqrt(2) 0.45 u; the relative bound at the threshold is 5 standard deviations
over rho_thr, and never looser than the workload's 1e-3 for FP16."""

import math

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O
from oracle import quant_oracle as Q
from tests.parity import compare_triggers, oracle_rho2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
KINDS = {"f16": 1, "bf16": 2}


def snr_tol(kind, thr):
    t = 5 * math.sqrt(2) * 0.45 * Q.UNIT_ROUNDOFF[kind] / thr
    return min(t, 1e-3) if kind == "f16" else t


@pytest.fixture(scope="module")
def mf(lib):
    from paper_2309_00019_gb300 import mf as m
    return m


def _pack16(stored, kind):
    """Oracle-stored complex values -> uint32 words (real in the low half)."""
    if kind == "f16":
        re = stored.real.astype(np.float16).view(np.uint16).astype(np.uint32)
        im = stored.imag.astype(np.float16).view(np.uint16).astype(np.uint32)
    else:
        re = (stored.real.astype(np.float32).view(np.uint32) >> 16).astype(np.uint32)
        im = (stored.imag.astype(np.float32).view(np.uint32) >> 16).astype(np.uint32)
    return np.ascontiguousarray(re | (im << 16))


@pytest.mark.parametrize("kind", list(KINDS))
def test_device_quantiser_matches_oracle_rounding(mf, kind):
    c = synth.make_config1()
    bank = c.bank()
    p = mf.Plan(c.fs, c.n, 1, c.f_low, c.f_high, c.thr, c.window, dtype=KINDS[kind])
    p.set_psd(c.psd)
    p.bank_reserve(len(bank), KINDS[kind])
    p.bank_quantize_rows(0, torch.from_numpy(bank).to(DEV))
    st, s = Q.quantize_rows(bank, kind)
    # the oracle's stored values and scales loaded directly: identical bank
    p2 = mf.Plan(c.fs, c.n, 1, c.f_low, c.f_high, c.thr, c.window, dtype=KINDS[kind])
    p2.set_psd(c.psd)
    p2.load_bank(_pack16(st, kind), dtype=KINDS[kind], scales=s.astype(np.float32))
    assert np.array_equal(p.sigmasq(), p2.sigmasq())
    w = O.weights(c.n, c.fs, c.f_low, c.f_high, c.psd)
    assert np.allclose(p.sigmasq(), O.sigmasq(st * s[:, None], w), rtol=1e-12, atol=0)
    # host staging gives the same bank
    p3 = mf.Plan(c.fs, c.n, 1, c.f_low, c.f_high, c.thr, c.window, dtype=KINDS[kind])
    p3.set_psd(c.psd)
    p3.bank_reserve(len(bank), KINDS[kind])
    p3.bank_quantize_rows(0, bank)
    assert np.array_equal(p3.sigmasq(), p.sigmasq())


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("data16", [False, True])
def test_config1_16bit_against_fp64_oracle(mf, kind, data16):
    c = synth.make_config1()
    bank = c.bank()
    sfd = (c.noise_fd + c.signal_fd).astype(np.complex64)
    p = mf.Plan(c.fs, c.n, 1, c.f_low, c.f_high, c.thr, c.window, dtype=KINDS[kind])
    p.set_psd(c.psd)
    p.bank_reserve(len(bank), KINDS[kind])
    p.bank_quantize_rows(0, bank)
    if data16:
        p.set_data_dtype(KINDS[kind])
    p.filter(torch.from_numpy(sfd[None, :]).to(DEV))
    trig, n, _ = p.triggers()
    rho2, z = oracle_rho2(sfd.astype(np.complex128), bank.astype(np.complex128), c.psd, c.n, c.fs, c.f_low, c.f_high)
    tol = snr_tol(kind, c.thr) if data16 else snr_tol(kind, c.thr) / math.sqrt(2)
    st = compare_triggers(trig, rho2, np.arange(len(bank)), c.thr, c.window, rel_tie=4 * tol, snr_rtol=tol)
    print(f"\nconfig 1 {kind} bank, {'16-bit' if data16 else 'FP32'} data: {n} triggers, max rel SNR err "
          f"{st['max_rel_snr']:.2e} (bound {tol:.1e}), window-edge differences {st['edge']}")
    inj = trig[(trig["tmpl"] == c.inj_tmpl) & (trig["sample"] // c.window == c.inj_sample // c.window)]
    assert len(inj) == 1 and abs(int(inj["sample"][0]) - c.inj_sample) <= 1


def test_16bit_data_needs_matching_bank(mf):
    c = synth.make_config1()
    p = mf.Plan(c.fs, c.n, 1, c.f_low, c.f_high, c.thr, c.window)
    p.set_psd(c.psd)
    p.load_bank(c.bank())
    p.set_data_dtype(1)
    sfd = torch.from_numpy((c.noise_fd + c.signal_fd).astype(np.complex64)[None, :]).to(DEV)
    with pytest.raises(mf.MFError):
        p.filter(sfd)
    p.set_data_dtype(0)
    p.filter(sfd)
    with pytest.raises(mf.MFError):
        p.bank_quantize_rows(0, c.bank())  # an FP32 bank has nothing to quantise into


def _keys(t, n_tmpl, window):
    return (t["det"].astype(np.int64) * n_tmpl + t["tmpl"]) * (1 << 12) + t["sample"] // window


def test_config4_full_bank_16bit_vs_fp32_and_oracle(mf):
    """50,000 templates x 2 detectors x 256 s at 4096 Hz (N = 2^20): every
    precision filters the whole bank in the default launch configuration (FP32,
    FP16 and bfloat16 storage of bank and data; FP32 and FP16 banks with the FP16
    intermediate and the tensor-core row pass); the FP32 CUDA path is the
    reference for the trigger sets, and the FP64 oracle checks a sample of
    templates one by one."""
    c = synth.make_config4()
    n, nb, nt = c.n, c.n // 2 + 1, len(c.m1)
    ld = (nb + 63) // 64 * 64
    d = c.data_fd(DEV, ld=ld)
    # oracle sample: the templates closest in chirp times to 6 injections, plus 6 random ones
    tau = np.stack(synth.chirp_times(c.m1, c.m2, c.f_low), axis=1)
    rng = np.random.default_rng(9)
    ids = []
    for i in rng.choice(len(c.inj["m1"]), 6, replace=False):
        ti = np.array(synth.chirp_times(c.inj["m1"][i], c.inj["m2"][i], c.f_low))
        ids.append(int(np.argmin(((tau - ti) / tau.std(axis=0)) ** 2 @ np.ones(2))))
    ids = sorted(set(ids) | set(int(x) for x in rng.choice(nt, 6, replace=False)))
    res, ms = {}, {}
    # (bank and data storage, FP16 pass-1 -> pass-2 intermediate with the tensor-core row pass); the "-tc" forms
    # keep FP32 weighted data, which the FP16 intermediate needs
    kinds = {"f32": (0, False), "f16": (1, False), "bf16": (2, False), "f32-tc": (0, True), "f16-tc": (1, True)}
    for kind, (dt, tc) in kinds.items():
        p = mf.Plan(c.fs, n, 2, c.f_low, c.fs / 2, c.thr, c.window, dtype=dt, max_triggers=1 << 24)
        p.set_psd(c.psd)
        p.bank_reserve(nt, dt)
        for r0, rows in synth.taylorf2_chunks_torch(n, c.fs, c.m1, c.m2, c.f_low, DEV, chunk=1024, ld=ld):
            if dt == 0:
                p.bank_set_rows(r0, rows, ld=ld, on_device=1)
            else:
                p.bank_quantize_rows(r0, rows, ld=ld, on_device=1)
        if tc:
            p.set_intermediate(mf.MF_F16)
        elif dt:
            p.set_data_dtype(dt)
        p.filter(d, ld=ld)  # warm-up (tables, scales)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        p.filter(d, ld=ld)
        e1.record()
        e1.synchronize()
        ms[kind] = e0.elapsed_time(e1)
        trig, cnt, _ = p.triggers()
        assert cnt == len(trig)
        res[kind] = trig
        p.close()
        del p
        torch.cuda.empty_cache()
    sample_rows = synth.taylorf2_torch(n, c.fs, c.m1[ids], c.m2[ids], c.f_low, DEV).cpu().numpy()
    dh = d[:, :nb].cpu().numpy().astype(np.complex128)
    rho2, _ = oracle_rho2(dh, sample_rows.astype(np.complex128), c.psd, n, c.fs, c.f_low, c.fs / 2)
    ref = res["f32"]
    kref = _keys(ref, nt, c.window)
    for kind, (dt, tc) in kinds.items():
        # the FP16 intermediate's bound is the metric's 1e-3; an FP16 bank adds its storage bound
        if tc:
            tol = 1e-3 + (snr_tol("f16", c.thr) if dt else 0.0)
        else:
            tol = 1e-4 if kind == "f32" else snr_tol(kind, c.thr)
        tr = res[kind]
        sub = tr[np.isin(tr["tmpl"], ids)]
        st = compare_triggers(sub, rho2, ids, c.thr, c.window, rel_tie=4 * tol, snr_rtol=tol)
        tds = nt * 2 * (n / c.fs) / (ms[kind] * 1e-3)
        line = (f"\nconfig 4 {kind}: filter {ms[kind]:.1f} ms ({tds:.3g} template-s/s), {len(tr)} triggers; "
                f"oracle sample ({len(ids)} templates, "
                f"{st['exact'] + st['tie_swaps']} triggers): max rel SNR err {st['max_rel_snr']:.2e} (bound {tol:.1e})")
        if kind != "f32":
            k = _keys(tr, nt, c.window)
            common, ia, ib = np.intersect1d(kref, k, return_indices=True)
            rel = np.abs(tr["snr"][ib].astype(np.float64) - ref["snr"][ia]) / ref["snr"][ia]
            only_ref = np.setdiff1d(np.arange(len(ref)), ia)
            only_new = np.setdiff1d(np.arange(len(tr)), ib)
            # a window present in one set only sits at the threshold within the error bound
            edge = np.concatenate([ref["snr"][only_ref], tr["snr"][only_new]]).astype(np.float64)
            assert np.all(np.abs(edge - c.thr) <= 2 * tol * c.thr), edge.max(initial=0)
            assert rel.max() <= 2 * tol
            moved = int((tr["sample"][ib] != ref["sample"][ia]).sum())
            line += (f"; vs FP32 path: {len(common)} common windows, max rel SNR diff {rel.max():.2e}, "
                     f"{len(only_ref)} only in FP32, {len(only_new)} only in {kind}, {moved} peaks moved")
        print(line)
