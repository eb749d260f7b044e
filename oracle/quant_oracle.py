"""CPU oracle of reduced-precision storage (bank and weighted data).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module;
it shares no code with the CUDA path.

The paper filters in double precision on CPUs and has no reduced-precision
storage; the precision workload stores templates and weighted data in 16 bits
with a per-row scale and accumulates in 32 bits, with sigma^2 (Eq. 2) in
float64.  This module states that storage rule in numpy:

  * a row x (complex) gets the power-of-two scale s = 2^(e - 15), where
    max_k max(|Re x_k|, |Im x_k|) = m 2^e with m in [1/2, 1), so that the
    stored values x / s have a largest component in [2^14, 2^15);
  * the stored values are x / s rounded to nearest, ties to even, in IEEE
    binary16 (FP16) or in bfloat16 (the upper half of a binary32);
  * the template's sigma^2 and every product use the stored value times s.

The error model the tests pin: rounding to p significant bits has relative
error at most u = 2^-p (p = 11 for FP16, 8 for bfloat16), uniformly spread,
so a row's rounding error delta has |delta|^2 ~ |x|^2 u^2 / 3 (RMS relative
u / sqrt 3).  For a matched filter with sigma^2 of the stored template, only
the part of delta orthogonal to h changes rho, giving (i) a relative loss of
at most |delta|^2 / (2 |h|^2) for the exactly matching signal, and (ii) in
Gaussian noise an additive rho error with standard deviation about
|delta| / |h| = u / sqrt 3.
"""

from __future__ import annotations

import numpy as np

UNIT_ROUNDOFF = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}


def pow2_scale(amax):
    """s = 2^(e - 15) for amax = m 2^e, m in [1/2, 1); 1 for amax <= 0."""
    amax = np.asarray(amax, np.float64)
    _, e = np.frexp(np.where(amax > 0, amax, 1.0))
    s = np.ldexp(1.0, (e - 15).astype(np.int64))
    return np.where(amax > 0, s, 1.0)


def round_f16(x):
    """binary32 -> binary16, round to nearest even (IEEE, via numpy)."""
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float64)


def round_bf16(x):
    """binary32 -> bfloat16 (sign, 8 exponent bits, 7 fraction bits), round to
    nearest even on the dropped 16 bits; finite inputs only."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def quantize_rows(x, kind):
    """Stored values and scales of complex rows x [..., n] (binary32 input).

    Returns (stored complex128 [..., n], scale float64 [...]); the
    represented row is stored * scale."""
    x = np.asarray(x, np.complex64)
    rnd = round_f16 if kind == "f16" else round_bf16
    amax = np.maximum(np.abs(x.real), np.abs(x.imag)).max(axis=-1).astype(np.float64)
    s = pow2_scale(amax)
    inv = (1.0 / s)[..., None]
    re = rnd((x.real.astype(np.float64) * inv).astype(np.float32))
    im = rnd((x.imag.astype(np.float64) * inv).astype(np.float32))
    return re + 1j * im, s


def dequantize_rows(x, kind):
    """The row each stored 16-bit row represents (stored * scale), complex128."""
    st, s = quantize_rows(x, kind)
    return st * s[..., None]
