"""Pins of the oracle MLP (learned collide) against finite differences and closed forms."""
import math

import numpy as np
import pytest
from scipy.stats import norm

from oracle import mlp


def test_gelu_closed_forms():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 3.0])
    assert np.allclose(mlp.gelu(z), z * norm.cdf(z), rtol=1e-14, atol=1e-16)
    assert mlp.gelu(0.0) == 0.0 and mlp.gelu_grad(0.0) == pytest.approx(0.5)
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, atol=1e-15)
    h = 1e-6
    assert np.allclose((mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), mlp.gelu_grad(z), atol=1e-9)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(1, scale=1.5)
    x = rng.standard_normal((16, 37))
    t = rng.standard_normal((16, 37))
    loss, g = mlp.loss_grad(p, x, t)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    idx = np.concatenate([idx, [0, 4735, 4736, 4863, 4864, 21247, 21248, 21375, 21376, 26111, 26112, 26148]])
    h = 1e-6
    for k in idx:
        q = p.copy()
        q[k] += h
        lp = mlp.loss_grad(q, x, t)[0]
        q[k] -= 2 * h
        lm = mlp.loss_grad(q, x, t)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, abs(g[k])) + 1e-9, k


def test_pack_layout_and_bf16_rounding():
    assert mlp.NPARAM == 26149
    p = np.arange(mlp.NPARAM, dtype=np.float64)
    w = mlp.unpack(p)
    assert w["W1"][1, 0] == 37 and w["b1"][0] == 4736 and w["W2"][0, 1] == 4865
    assert w["W3"][36, 127] == 26111 and w["b3"][36] == 26148
    assert np.array_equal(mlp.pack(w), p)
    # bfloat16 keeps 8 significant bits, ties to even
    assert mlp.round_bf16(np.array([1.0 + 2**-8]))[0] == 1.0
    assert mlp.round_bf16(np.array([1.0 + 3 * 2**-8]))[0] == 1.0 + 2**-6
    assert mlp.round_bf16(np.array([1.0 + 2**-7]))[0] == 1.0 + 2**-7
