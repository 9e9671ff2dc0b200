"""Pin of the CPU oracle of the warm-start network: analytic gradients against central
finite differences (FP64), and the bfloat16 rounding against its bit-level definition."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    F, H = 5, 7
    rng = np.random.default_rng(0)
    theta = mlp.init_params(F, H, 1) + 0.05 * rng.normal(size=mlp.n_params(F, H))
    X = rng.normal(size=(9, F))
    T = rng.normal(size=(9, 2))
    loss, g = mlp.loss_and_grad(theta, F, H, X, T)
    eps = 1e-6
    fd = np.zeros_like(theta)
    for k in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        fd[k] = (mlp.loss_and_grad(tp, F, H, X, T)[0] - mlp.loss_and_grad(tm, F, H, X, T)[0]) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)
    # the loss is the mean squared error of the forward pass
    y, _ = mlp.forward(theta, F, H, X)
    assert abs(loss - np.sum((y - T) ** 2) / 9) < 1e-14


def test_bf16_rounding_definition():
    # values exactly representable in bfloat16 are kept; ties round to even; 8 significant bits
    assert mlp.bf16_round(np.float32(1.0)) == 1.0
    assert mlp.bf16_round(np.float32(1.0 + 2 ** -8)) == 1.0            # tie -> even (1.0)
    assert mlp.bf16_round(np.float32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6   # tie -> even (up)
    assert mlp.bf16_round(np.float32(1.0 + 2 ** -7)) == 1.0 + 2 ** -7
    x = np.random.default_rng(1).normal(size=1000).astype(np.float32)
    r = mlp.bf16_round(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8 + 1e-30)
