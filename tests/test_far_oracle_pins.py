"""Pins of the oracle's background estimate (CPU): Eq. (6)'s counting FAR on
hand-made backgrounds, the Sec. IV tail fit recovering a known exponential
tail, and the time-shifted background of Gaussian-noise triggers, whose
network-SNR tail follows from Appendix A (chi^2 with 2 dof per detector)."""

import math

import numpy as np
import pytest

from oracle import mf_oracle as O


def test_counting_far_closed_forms():
    bg = np.array([5.0, 6.0, 6.0, 7.5, 9.0])
    t_bg = 100.0
    # louder than every background value: 1 / T_b; ties count (>=)
    assert O.far_count([10.0], bg, t_bg)[0] == pytest.approx(1 / t_bg)
    assert O.far_count([9.0], bg, t_bg)[0] == pytest.approx(2 / t_bg)
    assert O.far_count([6.0], bg, t_bg)[0] == pytest.approx(5 / t_bg)
    assert O.far_count([1.0], bg, t_bg)[0] == pytest.approx(6 / t_bg)
    # scaled background volume
    assert O.far_count([6.0], bg, t_bg, scale=10.0)[0] == pytest.approx(41 / t_bg)


def test_tail_fit_recovers_an_exponential_tail():
    rng = np.random.default_rng(0)
    lam = 1.7
    bg = 6.0 + rng.exponential(1 / lam, 200000)  # n_b(x) = 2e5 exp(-lam (x - 6))
    alpha, beta = O.tail_fit(bg, 6.5)
    assert beta == pytest.approx(-lam, rel=0.03)
    assert alpha == pytest.approx(math.log(2e5) + 6.0 * lam, rel=0.02)
    # the fitted FAR extrapolates beyond the loudest background value
    fg = np.array([bg.max() + 2.0])
    f = O.far_fit(fg, alpha, beta, 1.0)[0]
    assert f == pytest.approx(1 + 2e5 * math.exp(-lam * (fg[0] - 6.0)), rel=0.2)
    assert O.far_count(fg, bg, 1.0)[0] == 1.0  # counting alone saturates at 1 / T_b


def test_time_shifted_gaussian_background_has_the_chi2_tail():
    """Independent detectors: shifted coincidences pair independent triggers;
    with per-trigger rho^2 ~ chi^2_2 conditioned on rho >= thr, the network
    rho_c^2 - 2 thr^2 is Gamma(2, 2), so the cumulative background at large
    rho_c^2 falls as (1 + x / 2) exp(-x / 2) with x = rho_c^2 - 2 thr^2."""
    rng = np.random.default_rng(1)
    thr = 2.0
    n = 400000
    r0 = thr ** 2 + rng.exponential(2.0, n)  # rho^2 of triggers above threshold (chi^2_2 tail)
    r1 = thr ** 2 + rng.exponential(2.0, n)
    rc2 = r0 + r1
    x = np.array([6.0, 10.0, 14.0])
    got = O.background_count(rc2, 2 * thr ** 2 + x) / n
    expect = (1 + x / 2) * np.exp(-x / 2)
    assert np.allclose(got, expect, rtol=0.05)
    # and the log-linear fit of the far tail has slope close to -1/2 in rho_c^2
    alpha, beta = O.tail_fit(rc2, 2 * thr ** 2 + 12.0)
    assert -0.6 < beta < -0.4
