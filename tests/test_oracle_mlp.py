"""Pins of the fp64 network oracle: finite differences, closed forms, library routines."""
import math

import numpy as np
import pytest

from oracle import mlp as M


def _rand_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, M.NPARAM)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    p = _rand_params(1)
    X = rng.normal(0, 1, (7, M.F))
    T = rng.normal(0, 1, 7)
    _, g = M.loss_and_grad(p, X, T)
    h = 1e-6
    for i in list(range(0, M.NPARAM, 97)) + [M.OFF_B3, M.OFF_W3, M.OFF_B2, M.OFF_B1, M.OFF_W2 + 5]:
        e = np.zeros(M.NPARAM)
        e[i] = h
        num = (M.loss_and_grad(p + e, X, T)[0] - M.loss_and_grad(p - e, X, T)[0]) / (2 * h)
        assert num == pytest.approx(g[i], rel=1e-5, abs=1e-9)


def test_forward_reduces_to_closed_form_when_hidden_weights_vanish():
    """W1 = W2 = 0: every row gives b3 + sum_j W3_j GELU(b2_j) (GELU(b1) is multiplied by 0)."""
    p = _rand_params(2)
    p[M.OFF_W1:M.OFF_B1] = 0
    p[M.OFF_W2:M.OFF_B2] = 0
    W1, b1, W2, b2, W3, b3 = M.unpack(p)
    want = b3 + sum(W3[j] * 0.5 * b2[j] * (1 + math.erf(b2[j] / math.sqrt(2))) for j in range(M.H))
    X = np.random.default_rng(3).normal(0, 1, (5, M.F))
    assert np.allclose(M.forward(p, X), want, rtol=1e-14)


def test_gelu_is_z_times_normal_cdf():
    from scipy.stats import norm
    z = np.linspace(-6, 6, 101)
    assert np.allclose(M.gelu(z), z * norm.cdf(z), rtol=1e-12, atol=1e-15)
    assert np.allclose(M.gelu_grad(z), norm.cdf(z) + z * norm.pdf(z), rtol=1e-12, atol=1e-15)


def test_bf16_rounding_matches_torch_and_ties_to_even():
    import torch
    rng = np.random.default_rng(5)
    w = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 1000), [0.0, -0.0, 1.0, -2.5]]).astype(np.float32)
    want = torch.from_numpy(w).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(w), want)
    one = np.float32(1.0)
    half_ulp = np.float32(2.0 ** -8)   # bf16 spacing at 1 is 2^-7
    assert M.bf16(np.array([one + half_ulp], np.float32))[0] == 1.0                       # tie -> even (1.0)
    # halfway between 1 + 2^-7 (odd mantissa) and 1 + 2^-6 (even): goes to the even one
    assert M.bf16(np.array([one + 3 * half_ulp], np.float32))[0] == 1.0 + 2.0 ** -6


def test_features_from_definition_on_a_small_graph():
    u = np.array([0, 0, 1, 2, 2, 2], np.uint32)
    v = np.array([0, 1, 1, 0, 1, 2], np.uint32)
    f = M.features(u, v, 3, 3)
    # U vertex 2: degree 3, neighbours V0 (deg 2), V1 (deg 3), V2 (deg 1)
    assert f[2, 0] == pytest.approx(math.log1p(3) / 8)
    assert f[2, 1] == pytest.approx(math.log1p(6) / 16)
    assert f[2, 2] == pytest.approx(math.log1p(3) / 16)
    assert f[2, 3] == pytest.approx(math.log1p(3) / 16)
    assert f[2, 4] == 0 and f[3 + 1, 4] == 1
    assert f[2, 5] == pytest.approx(math.log1p(3) / 16)
    # V vertex 1: degree 3, neighbours U0 (2), U1 (1), U2 (3)
    assert f[4, 1] == pytest.approx(math.log1p(6) / 16)
    assert f[4, 5] == pytest.approx(math.log1p(3) / 16)



def test_score_weights_equal_scores_give_the_full_unit():
    """exp(s - max s) = 1 for every vertex when all scores are equal: 2^24 each,
    whatever the common value (the maximum is subtracted before exp)."""
    for c in (-40.0, 0.0, 3.0, 700.0):
        w = M.score_weights(np.full(7, c))
        assert w.dtype == np.uint64
        assert np.all(w == 1 << 24)


def test_score_weights_halving_per_ln2():
    """s_i = s_max - k ln 2 gives 2^24 e^(-k ln 2) = 2^(24-k); the float64 exp may
    land one unit low before the floor, never more."""
    k = np.arange(0, 24)
    s = 5.0 - k * math.log(2.0)
    w = M.score_weights(s).astype(np.int64)
    want = (1 << (24 - k)).astype(np.int64)
    assert np.all(np.abs(w - want) <= 1)
    assert w[0] == 1 << 24


def test_score_weights_floor_not_round_and_floor_at_one():
    """A ratio of 0.3 gives floor(0.3 * 2^24) = 5033164 (rounding would give
    5033165); ratios below 2^-24 are lifted to 1, so every vertex can be drawn."""
    s = np.array([2.0, 2.0 + math.log(0.3), 2.0 - 17.0 * math.log(2.0), 2.0 - 30.0, -1e6])
    w = M.score_weights(s)
    assert w[0] == 1 << 24
    assert w[1] == 5033164
    assert w[2] in (127, 128)
    assert w[3] == 1 and w[4] == 1


def test_score_weights_depend_only_on_score_differences():
    """Shifting every score by a constant leaves the weights unchanged; without the
    max subtraction the shifted scores would clamp to 2^24 everywhere."""
    s = np.array([0.0, -1.0, -2.5, -0.25])
    w0 = M.score_weights(s)
    for c in (3.0, 50.0, -20.0):
        assert np.array_equal(M.score_weights(s + c), w0)
    assert w0[1] == math.floor(16777216.0 / math.e)
    assert np.all(np.diff(M.score_weights(np.array([0.0, -0.1, -0.2, -0.3])).astype(np.int64)) < 0)
