"""Pins of the ordering network's CPU reference (oracle/mlp.py).

The backward pass is pinned by central finite differences of the loss in
float64 without BF16 rounding; the BF16 rounding function is pinned against
torch's own float32 -> bfloat16 conversion (round to nearest, ties to even).
"""
import numpy as np
import torch

from oracle import mlp


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-6, 6, size=5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0, -3.3e-5]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = rng.normal(size=mlp.NPARAM) * 0.3
    X = rng.normal(size=(40, mlp.IN))
    T = rng.normal(size=40)
    g, _ = mlp.gradient(p, X, T, quantize=False)
    eps = 1e-6
    idx = rng.choice(mlp.NPARAM, size=200, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, 0, 16 * 64 + 3]])   # b3, W1[0,0], a b1 entry
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = eps
        lp = mlp.gradient(p + e, X, T, quantize=False)[1]
        lm = mlp.gradient(p - e, X, T, quantize=False)[1]
        num = (lp - lm) / (2 * eps)
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, g[i])


def test_quantised_network_stays_close_to_real_one():
    rng = np.random.default_rng(2)
    p = rng.normal(size=mlp.NPARAM) * 0.2
    X = rng.normal(size=(64, mlp.IN))
    y_q, _ = mlp.forward(p, X, quantize=True)
    y_r, _ = mlp.forward(p, X, quantize=False)
    assert np.max(np.abs(y_q - y_r)) <= 0.05 * (np.max(np.abs(y_r)) + 1e-3)
