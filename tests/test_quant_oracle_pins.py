"""Pins of the reduced-precision storage oracle (CPU): the rounding rules against
brute force and IEEE, the power-of-two scale rule, and the error model the
GPU precision tests take their tolerances from."""

import math

import numpy as np
import pytest

import synth
from oracle import mf_oracle as O
from oracle import quant_oracle as Q


def _nearest_even(x, grid_step_fn):
    """Brute force: the nearest of the two grid neighbours, ties to the one whose
    last significand bit is 0."""
    lo, hi, lsb_lo = grid_step_fn(x)
    if x - lo < hi - x:
        return lo
    if x - lo > hi - x:
        return hi
    return lo if lsb_lo == 0 else hi


def _bf16_neighbours(x):
    # x > 0 normal: significand grid of 8 bits in x's binade
    e = math.floor(math.log2(x))
    step = 2.0 ** (e - 7)
    k = math.floor(x / step)
    return k * step, (k + 1) * step, k & 1


def _f16_neighbours(x):
    e = math.floor(math.log2(x))
    step = 2.0 ** (e - 10)
    k = math.floor(x / step)
    return k * step, (k + 1) * step, k & 1


def test_rounding_matches_brute_force_nearest_even():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(1.0, 2.0, 2000), 2.0 ** rng.uniform(-10, 10, 2000)]).astype(np.float32)
    # exact ties of both formats
    ties16 = [1 + 2 ** -11, 1 + 3 * 2 ** -11, 3 + 2 ** -10, 1000 + 2 ** -2 * 0.5 * 2]
    ties_b = [1 + 2 ** -8, 1 + 3 * 2 ** -8, 5.0 + 2 ** -6, 2 ** 20 * (1 + 2 ** -8)]
    for x in list(xs) + [np.float32(t) for t in ties16]:
        assert Q.round_f16(x) == _nearest_even(float(x), _f16_neighbours), x
    for x in list(xs) + [np.float32(t) for t in ties_b]:
        assert Q.round_bf16(x) == _nearest_even(float(x), _bf16_neighbours), x
    # sign symmetry, representable values unchanged
    assert Q.round_bf16(np.float32(-1.5)) == -1.5 and Q.round_f16(np.float32(-1.5)) == -1.5
    assert Q.round_bf16(np.float32(1 + 2 ** -8)) == 1.0 and Q.round_bf16(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6


def test_relative_rounding_error_bounded_by_unit_roundoff():
    rng = np.random.default_rng(1)
    x = (2.0 ** rng.uniform(-10, 14, 100000) * rng.choice([-1, 1], 100000)).astype(np.float32)
    for kind, fn in (("f16", Q.round_f16), ("bf16", Q.round_bf16)):
        rel = np.abs(fn(x) - x.astype(np.float64)) / np.abs(x.astype(np.float64))
        u = Q.UNIT_ROUNDOFF[kind]
        assert rel.max() <= u * (1 + 1e-12)
        assert rel.max() > 0.9 * u  # the bound is attained (no hidden extra precision)


def test_pow2_scale_puts_row_maximum_in_binade_14():
    amax = 2.0 ** np.linspace(-60, 60, 997)
    s = Q.pow2_scale(amax)
    assert np.all(np.log2(s) == np.round(np.log2(s)))
    r = amax / s
    assert np.all((r >= 2.0 ** 14) & (r < 2.0 ** 15))
    assert Q.pow2_scale(0.0) == 1.0
    # FP16's largest finite value is 65504 > 2^15: no stored value overflows
    rng = np.random.default_rng(2)
    x = (rng.standard_normal((4, 300)) + 1j * rng.standard_normal((4, 300))) * 1e-21
    st, s = Q.quantize_rows(x, "f16")
    m = np.maximum(np.abs(st.real), np.abs(st.imag)).max(axis=1)
    assert np.all((m >= 2 ** 14) & (m <= 2 ** 15))


def _setup(n=16384, fs=512.0, f_low=30.0):
    psd = synth.psd_bins(n, fs)
    w = O.weights(n, fs, f_low, fs / 2, psd)
    h = synth.taylorf2(n, fs, 1.6, 1.3, f_low)
    return psd, w, h


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_exact_signal_loss_is_second_order(kind):
    """A noiseless injection of h filtered with the stored template (and its own
    sigma) loses at most |delta|^2 / (2 |h|^2) of rho (Cauchy-Schwarz bound)."""
    n, fs = 16384, 512.0
    psd, w, h = _setup(n, fs)
    hq = Q.dequantize_rows(h.astype(np.complex64), kind)
    h64 = h.astype(np.complex64).astype(np.complex128)
    sig = math.sqrt(O.sigmasq(h64, w))
    rho_exact = np.abs(O.complex_snr(h64, h64, w, n)).max() / sig
    rho_q = np.abs(O.complex_snr(h64, hq, w, n)).max() / math.sqrt(O.sigmasq(hq, w))
    d2 = O.sigmasq(hq - h64, w) / sig ** 2
    loss = 1 - rho_q / rho_exact
    assert rho_exact == pytest.approx(sig, rel=1e-12)
    assert -1e-12 <= loss <= 0.5 * d2 * (1 + 1e-6) + 1e-15
    assert d2 < Q.UNIT_ROUNDOFF[kind] ** 2  # RMS relative rounding below u


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_noise_rho_error_follows_the_rounding_norm(kind):
    """In Gaussian noise the rho error of the stored template has standard
    deviation |delta|_w / sigma (one quadrature of the rounding error)."""
    n, fs = 16384, 512.0
    psd, w, h = _setup(n, fs)
    rng = np.random.default_rng(3)
    h64 = h.astype(np.complex64).astype(np.complex128)
    hq = Q.dequantize_rows(h.astype(np.complex64), kind)
    sig, sigq = math.sqrt(O.sigmasq(h64, w)), math.sqrt(O.sigmasq(hq, w))
    pred = math.sqrt(O.sigmasq(hq - h64, w)) / sig
    errs = []
    for _ in range(4):
        s = synth.coloured_noise_fd(rng, n, fs)
        r = np.abs(O.complex_snr(s, h64, w, n)) / sig
        rq = np.abs(O.complex_snr(s, hq, w, n)) / sigq
        errs.append(rq - r)
    sd = float(np.std(np.concatenate(errs)))
    assert 0.8 * pred < sd < 1.25 * pred
    # and the model's size: RMS relative rounding of a few tenths of u
    assert 0.2 * Q.UNIT_ROUNDOFF[kind] < pred < 0.7 * Q.UNIT_ROUNDOFF[kind]
