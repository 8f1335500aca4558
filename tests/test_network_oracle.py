"""Pin of the network oracle: its backpropagated gradient equals central
finite differences of its own loss (FP64), and the loss is exactly zero when
the targets are the network's outputs."""
import numpy as np

from oracle.network import forward, loss_and_grad, param_count


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    H, P, nx = 6, 3, 7
    theta = 0.3 * rng.standard_normal(param_count(H))
    x = rng.standard_normal((P, nx, 26))
    t = rng.standard_normal((P, nx, 5))
    loss, g = loss_and_grad(theta, H, x, t)
    eps = 1e-6
    for i in rng.choice(theta.size, 40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (loss_and_grad(tp, H, x, t)[0] - loss_and_grad(tm, H, x, t)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i]))


def test_zero_loss_at_own_output_and_padding():
    rng = np.random.default_rng(1)
    H = 4
    theta = rng.standard_normal(param_count(H))
    x = rng.standard_normal((2, 5, 26))
    y, _ = forward(theta, H, x)
    loss, g = loss_and_grad(theta, H, x, y)
    assert loss == 0.0 and np.all(g == 0.0)
    # receptive field: changing cell 0 does not affect outputs beyond cell 4
    x2 = x.copy()
    x2[:, 0] += 1.0
    y2, _ = forward(theta, H, x2)
    assert np.array_equal(y2[:, 5:], y[:, 5:]) and not np.allclose(y2[:, :5], y[:, :5])
