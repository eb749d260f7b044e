"""GPU checks of gating (Sec. VI): the gate statistic and gate list found by the
library (a one-row sqrt(S_n) bank through mf_filter) against the FP64 oracle,
the windows applied by mf_gate_apply against the oracle's, and the effect on a
search: the glitch's triggers go, an injected chirp keeps its SNR."""

import math

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O
from tests.parity import compare_triggers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
N, FS, F_LOW = 1 << 16, 1024.0, 20.0


@pytest.fixture(scope="module")
def mf(lib):
    from paper_2309_00019_gb300 import mf as m
    return m


def _data(seed=4):
    rng = np.random.default_rng(seed)
    t = np.arange(N) / FS
    x = np.stack([synth.strain_from_fd(synth.coloured_noise_fd(rng, N, FS), N, FS) for _ in range(2)])
    a = synth.sine_gaussian_amplitude(400.0, 150.0, 6.0)
    x[0] += synth.sine_gaussian(t, 20.0, 150.0, 6.0, a, 0.0)
    x[1] += synth.sine_gaussian(t, 41.3, 90.0, 9.0, 0.7 * a, 1.1)
    psd = synth.psd_bins(N, FS)
    w = O.weights(N, FS, F_LOW, FS / 2, psd)
    h = synth.taylorf2(N, FS, 14.0, 11.0, F_LOW)
    amp = 15.0 / math.sqrt(O.sigmasq(h, w))
    x[0] += synth.strain_from_fd(synth.taylorf2(N, FS, 14.0, 11.0, F_LOW, t0=50.0, amp=amp), N, FS)
    return x.astype(np.float32), psd, h


def _gate_plan(mf, psd, thr):
    p = mf.Plan(FS, N, 2, F_LOW, FS / 2, thr, int(FS), max_triggers=1 << 16)
    p.set_psd(psd)
    p.load_gate_template()
    return p


def _spectra(mf, p, x_dev):
    dt = torch.zeros((2, N // 2 + 1), dtype=torch.complex64, device=DEV)
    p.strain_to_fd(x_dev, dt)
    return dt


@pytest.mark.parametrize("thr", [3.0, 30.0])
def test_gates_match_the_oracle_statistic(mf, thr):
    """thr 3: a gate in almost every window of noise (the statistic's parity); thr 30: the two glitches."""
    x, psd, _ = _data()
    p = _gate_plan(mf, psd, thr)
    p.filter(_spectra(mf, p, torch.from_numpy(x).to(DEV)))
    gates, n, _ = p.triggers()
    rho_g = O.gate_statistic(O.strain_to_fd(x.astype(np.float64), FS), psd, N, FS, F_LOW, FS / 2)
    st = compare_triggers(gates, (rho_g ** 2)[:, None, :], [0], thr, int(FS))
    if thr > 10:
        assert n == len(gates) >= 2
        for d, t0 in ((0, 20.0), (1, 41.3)):
            assert np.abs(gates["sample"][gates["det"] == d] / FS - t0).min() < 0.05
    else:
        assert n > 0.9 * 2 * (N // int(FS))
    print(f"\nthreshold {thr}: {n} gates, {st}")


def test_gate_apply_matches_the_oracle_window(mf):
    x, psd, _ = _data()
    p = _gate_plan(mf, psd, 30.0)
    xd = torch.from_numpy(x).to(DEV)
    p.filter(_spectra(mf, p, xd))
    gates, n, _ = p.triggers()
    assert n >= 2
    out = mf.gate_apply(xd, p, 0.25, 0.25)
    ref = O.gate_apply(x.astype(np.float64), FS, gates, 0.25, 0.25)
    got = out.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-6 * np.max(np.abs(x))
    for d in range(2):
        c = gates["sample"][gates["det"] == d]
        near = np.min(np.abs(np.arange(N)[:, None] - c[None, :]), axis=1) <= int(0.25 * FS)
        assert np.all(got[d][near] == 0.0)
    # in place, and no gates (a threshold nothing reaches) leaves the data unchanged
    xd2 = xd.clone()
    mf.gate_apply(xd2, p, 0.25, 0.25, out=xd2)
    assert torch.equal(xd2, out)
    q = _gate_plan(mf, psd, 1e4)
    q.filter(_spectra(mf, q, xd))
    assert q.triggers()[1] == 0
    assert torch.equal(mf.gate_apply(xd, q, 0.25, 0.25), xd)


def test_gating_removes_glitch_triggers_and_keeps_a_chirp(mf):
    x, psd, h = _data()
    xd = torch.from_numpy(x).to(DEV)
    g = _gate_plan(mf, psd, 30.0)
    g.filter(_spectra(mf, g, xd))
    xg = mf.gate_apply(xd, g, 0.25, 0.25)
    rng = np.random.default_rng(8)
    m1, m2 = synth.sample_bank_uniform_masses(rng, 12, 5.0, 20.0)
    m1 = np.append(m1, 14.0)
    m2 = np.append(m2, 11.0)
    bank = synth.taylorf2_torch(N, FS, m1, m2, F_LOW, DEV)
    res = {}
    for name, data in (("raw", xd), ("gated", xg)):
        p = mf.Plan(FS, N, 2, F_LOW, FS / 2, 6.0, int(FS), max_triggers=1 << 20)
        p.set_psd(psd)
        p.load_bank(bank)
        p.filter(_spectra(mf, p, data))
        res[name] = p.triggers()[0]
    raw, gated = res["raw"], res["gated"]
    near = lambda t, d, t0: t[(t["det"] == d) & (np.abs(t["sample"] / FS - t0) < 1.5)]
    assert len(near(raw, 0, 20.0)) > 0 and len(near(raw, 1, 41.3)) > 0  # the glitches ring the bank
    assert len(near(gated, 0, 20.0)) == 0 and len(near(gated, 1, 41.3)) == 0
    inj = lambda t: t[(t["det"] == 0) & (t["tmpl"] == len(m1) - 1) & (np.abs(t["sample"] / FS - 50.0) < 0.05)]
    a, b = inj(raw), inj(gated)  # the peak sits on a window edge: take the louder of the two windows
    assert len(a) >= 1 and len(b) >= 1
    ra, rb = float(a["snr"].max()), float(b["snr"].max())
    assert abs(rb / ra - 1) < 0.02
    print(f"\nraw {len(raw)} triggers, gated {len(gated)}; injection SNR {ra:.2f} -> {rb:.2f}")


def test_gate_apply_rejects_bad_arguments(mf):
    x, psd, _ = _data()
    p = _gate_plan(mf, psd, 30.0)
    xd = torch.from_numpy(x).to(DEV)
    p.filter(_spectra(mf, p, xd))
    with pytest.raises(mf.MFError):
        mf.gate_apply(xd, p, 0.25, -1.0)
    q = mf.Plan(FS, N, 2, F_LOW, FS / 2, 5.0, int(FS))
    with pytest.raises(mf.MFError):
        q.load_gate_template()  # no PSD yet
