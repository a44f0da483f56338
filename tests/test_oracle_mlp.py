"""Pins of the FP64 surrogate-MLP reference: finite differences and closed forms."""
import numpy as np

from oracle import mlp as M


def _setup(nin=3, H=5, nout=4, B=7, seed=0):
    rng = np.random.default_rng(seed)
    n = H * nin + H + H * H + H + nout * H + nout
    theta = rng.normal(scale=0.5, size=n)
    X = rng.uniform(-2, 3, size=(B, nin))
    T = rng.normal(size=(B, nout))
    lo, hi = np.full(nin, -2.0), np.full(nin, 3.0)
    ym, ys = rng.normal(size=nout), rng.uniform(0.5, 2.0, size=nout)
    return theta, X, T, lo, hi, ym, ys, nin, H, nout


def test_gradient_matches_central_differences():
    theta, X, T, lo, hi, ym, ys, nin, H, nout = _setup()
    _, g = M.loss_and_grad(theta, X, T, lo, hi, ym, ys, nin, H, nout)
    eps = 1e-6
    num = np.empty_like(theta)
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        num[i] = (M.loss_and_grad(tp, X, T, lo, hi, ym, ys, nin, H, nout)[0]
                  - M.loss_and_grad(tm, X, T, lo, hi, ym, ys, nin, H, nout)[0]) / (2 * eps)
    np.testing.assert_allclose(g, num, rtol=1e-6, atol=1e-9)


def test_silu_derivative_and_values():
    z = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(M.silu_grad(z), (M.silu(z + 1e-6) - M.silu(z - 1e-6)) / 2e-6, rtol=1e-6, atol=1e-9)
    assert M.silu(0.0) == 0.0 and abs(M.silu(50.0) - 50.0) < 1e-12


def test_zero_hidden_weights_give_bias_output_and_mean_gradient():
    # W3 = 0: y = b3 for every input, so d loss/d b3 = mean_batch(b3 - t)/n_out
    theta, X, T, lo, hi, ym, ys, nin, H, nout = _setup(seed=3)
    W1, b1, W2, b2, W3, b3 = M.split(theta, nin, H, nout)
    n3 = nout * H
    off_W3 = H * nin + H + H * H + H
    theta[off_W3:off_W3 + n3] = 0.0
    f = M.forward(theta, X, lo, hi, nin, H, nout)
    np.testing.assert_allclose(f["Y"], np.tile(b3, (X.shape[0], 1)))
    _, g = M.loss_and_grad(theta, X, T, lo, hi, ym, ys, nin, H, nout)
    t = (T - ym) / ys
    np.testing.assert_allclose(g[-nout:], (b3 - t).mean(0) / nout, rtol=1e-12)
    # and the hidden layers receive no gradient through W3 = 0
    assert np.all(g[:off_W3] == 0.0)


def test_input_scaling_maps_bounds_to_unit_interval():
    theta, X, T, lo, hi, ym, ys, nin, H, nout = _setup()
    f = M.forward(theta, np.vstack([lo, hi]), lo, hi, nin, H, nout)
    np.testing.assert_allclose(f["Xn"], [[-1.0] * nin, [1.0] * nin])


def test_gradient_magnitude_bounds_and_positive_case():
    # |g| <= magnitude element by element on a random network; with every
    # weight, bias and scaled input positive and every output above its
    # target, no term of any gradient sum is negative, so the two coincide
    theta, X, T, lo, hi, ym, ys, nin, H, nout = _setup(seed=5)
    _, g = M.loss_and_grad(theta, X, T, lo, hi, ym, ys, nin, H, nout)
    mag = M.grad_magnitude(theta, X, T, lo, hi, ym, ys, nin, H, nout)
    assert np.all(mag >= np.abs(g) - 1e-15)
    assert np.any(mag > np.abs(g) * (1 + 1e-6))          # cancellation does occur
    rng = np.random.default_rng(6)
    theta = rng.uniform(0.1, 1.0, size=theta.size)
    X = rng.uniform(0.6, 3.0, size=X.shape)              # above the midpoint 0.5 of [-2, 3]: scaled input > 0
    T = np.full(T.shape, -1e3)
    _, g = M.loss_and_grad(theta, X, T, lo, hi, ym, ys, nin, H, nout)
    mag = M.grad_magnitude(theta, X, T, lo, hi, ym, ys, nin, H, nout)
    assert np.all(g > 0)
    np.testing.assert_allclose(mag, g, rtol=1e-12)
