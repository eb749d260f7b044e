"""Pins of the FP64 learned-proposal oracle: central finite differences of
the loss, closed forms of the masked cross-entropy, GELU against its
definition, and AdamW's first step."""

import math

import numpy as np
import pytest
from scipy import stats

from oracle import mlp_oracle as M

DIMS = (5, 16, 4, 12)  # n_in, width, depth, n_out (small copy of 5 -> 256 x4 -> 2000)


def test_param_count_of_the_workload_network():
    assert M.num_params(5, 256, 4, 2000) == 5 * 256 + 256 + 3 * (256 * 256 + 256) + 256 * 2000 + 2000


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = M.init_params(rng, DIMS)
    x = rng.standard_normal((7, DIMS[0]))
    nv = np.array([12, 3, 5, 1, 12, 7, 9])
    lab = np.array([2, 0, 4, 0, 11, 6, 8])
    loss, g = M.loss_and_grad(theta, x, nv, lab, DIMS)
    idx = rng.choice(len(theta), 60, replace=False)
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = 1e-6
        lp, _ = M.loss_and_grad(theta + e, x, nv, lab, DIMS)
        lm, _ = M.loss_and_grad(theta - e, x, nv, lab, DIMS)
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_masked_ce_closed_forms():
    # equal logits: loss = log(n_valid); invalid slots carry no gradient
    logits = np.zeros((3, 10))
    loss, g = M.masked_ce(logits, np.array([1, 4, 10]), np.array([0, 3, 9]))
    assert loss == pytest.approx((0 + math.log(4) + math.log(10)) / 3)
    assert np.all(g[1, 4:] == 0) and np.all(g[0, 1:] == 0)
    assert g[0, 0] == pytest.approx(0.0)
    assert g.sum(axis=1) == pytest.approx(np.zeros(3), abs=1e-15)
    # huge values in invalid slots do not change the loss
    l2 = logits.copy()
    l2[1, 5] = 1e6
    assert M.masked_ce(l2, np.array([1, 4, 10]), np.array([0, 3, 9]))[0] == pytest.approx(loss)


def test_gelu_definition():
    z = np.linspace(-5, 5, 101)
    assert np.allclose(M.gelu(z), z * stats.norm.cdf(z), rtol=1e-12, atol=1e-15)
    h = 1e-6
    assert np.allclose(M.gelu_grad(z), (M.gelu(z + h) - M.gelu(z - h)) / (2 * h), atol=1e-8)


def test_adamw_first_step_is_sign_scaled_lr():
    theta = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -0.1, 2.0])
    th, m, v = M.adamw(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0, wd=0.0)
    assert np.allclose(th, theta - 0.01 * np.sign(g))
    th2, _, _ = M.adamw(theta, np.zeros(3), np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-8, wd=0.1)
    assert np.allclose(th2, theta * (1 - 0.01 * 0.1))


def test_topk_respects_mask_and_ties():
    logits = np.array([[1.0, 3.0, 3.0, 9.0], [5.0, 1.0, 0.0, 0.0]])
    out = M.topk_valid(logits, np.array([3, 1]), 2)
    assert out.tolist() == [[1, 2], [0, -1]]


def test_probability_mass_proposal_hand_cases():
    # logits ln(0.6), ln(0.3), ln(0.1) (plus an invalid slot): probabilities 0.6, 0.3, 0.1
    logits = np.log(np.array([[0.3, 0.6, 0.1, 50.0]]))
    nv = np.array([3])
    assert M.propose_mass(logits, nv, 4, 0.5).tolist() == [[1, -1, -1, -1]]
    assert M.propose_mass(logits, nv, 4, 0.85).tolist() == [[1, 0, -1, -1]]
    assert M.propose_mass(logits, nv, 4, 0.95).tolist() == [[1, 0, 2, -1]]
    assert M.propose_mass(logits, nv, 2, 0.95).tolist() == [[1, 0]]   # k caps it
    # p_mass >= 1 is the plain top-k; an empty neighbourhood proposes nothing
    rng = np.random.default_rng(0)
    l = rng.standard_normal((20, 9))
    n = rng.integers(0, 10, 20)
    assert (M.propose_mass(l, n, 4, 2.0) == M.topk_valid(l, n, 4)).all()
    assert (M.propose_mass(l, np.zeros(20, int), 3, 0.5) == -1).all()
