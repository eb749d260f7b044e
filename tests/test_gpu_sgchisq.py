"""GPU checks of the sine-Gaussian veto of heavy templates (Sec. III, chi^2_sg
and rho-hat of Eq. 3): the reduced statistic of every trigger of a template above
30 solar masses against the FP64 oracle, pass-through for lighter templates
and below snr_min, a broadband glitch that the veto cuts and a chirp that it
keeps."""

import math

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
N, FS, F_LOW = 1 << 16, 2048.0, 30.0
OFFSETS = [15.0, 30.0, 45.0, 60.0, 75.0, 90.0, 105.0, 120.0]


@pytest.fixture(scope="module")
def mf(lib):
    from paper_2309_00019_gb300 import mf as m
    return m


def _case(mf, dtype=0):
    rng = np.random.default_rng(12)
    m1 = np.array([25.0, 40.0, 6.0, 18.0])
    m2 = np.array([20.0, 30.0, 5.0, 10.0])  # total masses 45, 70, 11, 28: two heavy, two light
    psd = synth.psd_bins(N, FS)
    w = O.weights(N, FS, F_LOW, FS / 2, psd)
    f_final = synth.f_isco(m1, m2)
    t = np.arange(N) / FS
    fd = np.stack([synth.coloured_noise_fd(rng, N, FS) for _ in range(2)])
    a = synth.sine_gaussian_amplitude(60.0, float(f_final[0]), 3.0)
    fd[0] += O.strain_to_fd(synth.sine_gaussian(t, 10.0, float(f_final[0]), 3.0, a, 0.4), FS)
    h1 = synth.taylorf2(N, FS, m1[1], m2[1], F_LOW)
    fd[0] += synth.taylorf2(N, FS, m1[1], m2[1], F_LOW, t0=20.0, amp=12.0 / math.sqrt(O.sigmasq(h1, w)))
    strain = np.stack([synth.strain_from_fd(fd[d], N, FS) for d in range(2)]).astype(np.float32)
    bank = synth.taylorf2_torch(N, FS, m1, m2, F_LOW, DEV)
    p = mf.Plan(FS, N, 2, F_LOW, FS / 2, 3.0, int(FS), dtype=dtype, max_triggers=1 << 16)
    p.set_psd(psd)
    if dtype == 0:
        p.load_bank(bank)
    else:
        p.bank_reserve(len(m1), dtype)
        p.bank_quantize_rows(0, bank, ld=bank.shape[1], on_device=1)
        p.set_data_dtype(dtype)
    dt = torch.zeros((2, N // 2 + 1), dtype=torch.complex64, device=DEV)
    p.strain_to_fd(torch.from_numpy(strain).to(DEV), dt)
    p.filter(dt)
    trig, n, _ = p.triggers()
    cap = p.desc.max_triggers
    chi2 = torch.zeros(cap, dtype=torch.float32, device=DEV)
    newsnr = torch.zeros(cap, dtype=torch.float32, device=DEV)
    p.chisq(16, chi2, newsnr)
    s = O.strain_to_fd(strain.astype(np.float64), FS)
    return p, trig, n, newsnr, s, w, m1 + m2, f_final


def _run_sg(mf, p, f_final, mtotal, snr_in, snr_min=0.0):
    cap = p.desc.max_triggers
    c2 = torch.full((cap,), -1.0, dtype=torch.float32, device=DEV)
    hat = torch.full((cap,), -1.0, dtype=torch.float32, device=DEV)
    p.sgchisq(torch.tensor(f_final, dtype=torch.float32, device=DEV),
              torch.tensor(mtotal, dtype=torch.float32, device=DEV), snr_in, c2, hat, m_min=30.0, snr_min=snr_min,
              offsets=OFFSETS, q=20.0)
    torch.cuda.synchronize()
    return c2.cpu().numpy(), hat.cpu().numpy()


@pytest.mark.parametrize("dtype", [0, 1])
def test_sgchisq_matches_the_oracle(mf, dtype):
    p, trig, n, newsnr, s, w, mtotal, f_final = _case(mf, dtype)
    c2, hat = _run_sg(mf, p, f_final, mtotal, newsnr)
    ns = newsnr.cpu().numpy()[:n]
    heavy = mtotal[trig["tmpl"]] > 30.0
    assert heavy.sum() > 20 and (~heavy).sum() > 20
    # light templates pass through
    assert np.all(c2[:n][~heavy] == 0.0) and np.array_equal(hat[:n][~heavy], ns[~heavy])
    # heavy templates against the oracle (a sample of at most 150 triggers)
    idx = np.nonzero(heavy)[0]
    idx = idx[np.linspace(0, len(idx) - 1, min(150, len(idx))).astype(int)]
    tol = 2e-4 if dtype == 0 else 3e-3
    worst = 0.0
    for i in idx:
        t = trig[i]
        ref, used = O.sg_chisq(s[int(t["det"])], w, N, FS, int(t["sample"]), float(f_final[int(t["tmpl"])]),
                               OFFSETS, 20.0, FS / 2)
        assert used == 8
        err = abs(c2[i] - ref) / max(ref, 1e-3)
        worst = max(worst, err)
        assert err <= tol, (i, c2[i], ref)
        assert hat[i] == pytest.approx(float(O.sg_newsnr(ns[i], c2[i])), rel=1e-6)
    print(f"\n{'FP32' if dtype == 0 else 'FP16'} data: {len(idx)} heavy-template triggers, max rel chi2_r err {worst:.2e}")


def test_sgchisq_cuts_the_glitch_keeps_the_chirp_and_honours_snr_min(mf):
    p, trig, n, newsnr, s, w, mtotal, f_final = _case(mf)
    c2, hat = _run_sg(mf, p, f_final, mtotal, newsnr)
    ns = newsnr.cpu().numpy()[:n]
    g = np.nonzero((trig["det"] == 0) & (trig["tmpl"] == 0) & (np.abs(trig["sample"] / FS - 10.0) < 0.5))[0]
    gi = g[np.argmax(trig["snr"][g])]
    assert trig["snr"][gi] > 15.0 and c2[gi] > 20.0 and hat[gi] < 0.3 * ns[gi]
    c = np.nonzero((trig["det"] == 0) & (trig["tmpl"] == 1) & (np.abs(trig["sample"] / FS - 20.0) < 0.05))[0]
    ci = c[np.argmax(trig["snr"][c])]
    assert trig["snr"][ci] > 9.0 and c2[ci] < 6.0 and hat[ci] == ns[ci]
    # Eq. (3) on the glitch: rho^ = rho~ / sqrt(chi^2_sg)
    assert hat[gi] == pytest.approx(ns[gi] / math.sqrt(c2[gi]), rel=1e-6)
    # above every trigger's snr: nothing is vetoed
    c2b, hatb = _run_sg(mf, p, f_final, mtotal, newsnr, snr_min=1e9)
    assert np.all(c2b[:n] == 0.0) and np.array_equal(hatb[:n], ns)
    with pytest.raises(mf.MFError):
        p.sgchisq(newsnr, newsnr, newsnr, newsnr, newsnr, offsets=[], q=20.0)
