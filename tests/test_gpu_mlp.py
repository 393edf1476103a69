"""BF16 tensor-core forward/backward kernels of the ordering network vs the
float64 CPU reference with the same rounding points.

Tolerance: BF16 keeps 8 significant bits; the reference rounds the same
operands, so the remaining differences are FP32-vs-FP64 accumulation and the
occasional activation that rounds to the neighbouring BF16 value.  Every
parameter block must agree to 1e-2 of its own norm, outputs to 1e-2 of their
scale.
"""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu

BLOCKS = [("W1", 0, 1024), ("b1", 1024, 1088), ("W2", 1088, 5184), ("b2", 5184, 5248),
          ("w3", 5248, 5312), ("b3", 5312, 5313)]


@pytest.fixture(scope="module")
def ctx():
    from paper_1912_08453_gb300 import ccpm
    return ccpm.Context(0)


def test_param_layout(ctx):
    from paper_1912_08453_gb300 import ccpm
    assert ccpm.MLP_PARAMS == ref.NPARAM == BLOCKS[-1][2]


@pytest.mark.parametrize("B", [1, 63, 64, 200, 1000])
def test_forward_and_gradient_match_reference(ctx, B):
    from paper_1912_08453_gb300 import ccpm
    rng = np.random.default_rng(B)
    net = ccpm.Mlp(ctx, seed=B)
    p = net.params().astype(np.float64)
    p[1024:1088] = rng.normal(size=64) * 0.1          # non-zero biases
    p[5184:5248] = rng.normal(size=64) * 0.1
    p[5312] = 0.3
    net.set_params(p.astype(np.float32))
    p = net.params().astype(np.float64)
    X = rng.normal(size=(B, 16)).astype(np.float32)
    T = rng.normal(size=B).astype(np.float32)
    y = net.forward(X)
    y_ref, _ = ref.forward(p, X.astype(np.float64))
    assert np.max(np.abs(y - y_ref)) <= 1e-2 * (np.max(np.abs(y_ref)) + 1e-3)
    g, loss = net.gradient(X, T)
    g_ref, loss_ref = ref.gradient(p, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-2 * (abs(loss_ref) + 1e-6)
    for name, a, b in BLOCKS:
        err = np.linalg.norm(g[a:b] - g_ref[a:b])
        assert err <= 1e-2 * (np.linalg.norm(g_ref[a:b]) + 1e-7), (name, err, np.linalg.norm(g_ref[a:b]))


def test_training_fits_a_smooth_target(ctx):
    from paper_1912_08453_gb300 import ccpm
    rng = np.random.default_rng(7)
    X = rng.normal(size=(4096, 16)).astype(np.float32)
    t = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * X[:, 3]).astype(np.float32)
    net = ccpm.Mlp(ctx, seed=3)
    _, loss0 = net.gradient(X, t)
    net.train(X, t, steps=600, batch=256, lr=3e-3, seed=11)
    _, loss1 = net.gradient(X, t)
    assert loss1 < 0.25 * loss0, (loss0, loss1)
