"""FP64 reference of the surrogate MLP.  TEST INFRASTRUCTURE ONLY.

Only tests may import this module.  It restates, in plain numpy FP64, the
network the library trains: inputs scaled to [-1, 1] by per-input bounds,
n_in -> H -> H -> n_out with SiLU (z * sigmoid(z)) on the hidden layers,
mean-squared error 0.5 (y - t)^2 averaged over the batch and the outputs on
standardised targets t = (T - mean) / std, and its exact gradient by the
chain rule.  Flat parameter layout: W1[H][n_in] b1[H] W2[H][H] b2[H]
W3[n_out][H] b3[n_out].  Pinned by finite differences and closed forms.

``grad_magnitude`` gives, per parameter, the sum over the batch of the
absolute values of the terms whose signed sum is that gradient (the same
chain rule with |.| on every factor): the scale an element-by-element
comparison of a low-precision gradient is measured against.
"""
import numpy as np


def split(theta, nin, H, nout):
    o = 0
    out = []
    for shape in ((H, nin), (H,), (H, H), (H,), (nout, H), (nout,)):
        n = int(np.prod(shape))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape))
        o += n
    assert o == len(theta)
    return out


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(theta, X, x_lo, x_hi, nin, H, nout):
    W1, b1, W2, b2, W3, b3 = split(theta, nin, H, nout)
    Xn = 2.0 * (np.asarray(X, np.float64) - x_lo) / (np.asarray(x_hi) - np.asarray(x_lo)) - 1.0
    Z1 = Xn @ W1.T + b1
    H1 = silu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = silu(Z2)
    Y = H2 @ W3.T + b3
    return dict(Xn=Xn, Z1=Z1, H1=H1, Z2=Z2, H2=H2, Y=Y)


def loss_and_grad(theta, X, T, x_lo, x_hi, y_mean, y_std, nin, H, nout):
    """Returns (loss, flat gradient) in FP64."""
    W1, b1, W2, b2, W3, b3 = split(theta, nin, H, nout)
    f = forward(theta, X, x_lo, x_hi, nin, H, nout)
    t = (np.asarray(T, np.float64) - y_mean) / y_std
    B = f["Y"].shape[0]
    d = f["Y"] - t
    loss = 0.5 * np.mean(d * d)
    dY = d / (B * nout)
    gW3 = dY.T @ f["H2"]
    gb3 = dY.sum(0)
    dH2 = dY @ W3
    dZ2 = dH2 * silu_grad(f["Z2"])
    gW2 = dZ2.T @ f["H1"]
    gb2 = dZ2.sum(0)
    dH1 = dZ2 @ W2
    dZ1 = dH1 * silu_grad(f["Z1"])
    gW1 = dZ1.T @ f["Xn"]
    gb1 = dZ1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def grad_magnitude(theta, X, T, x_lo, x_hi, y_mean, y_std, nin, H, nout):
    """Per parameter: sum over samples of |term| of its gradient sum (flat,
    same layout as the gradient)."""
    W1, b1, W2, b2, W3, b3 = split(theta, nin, H, nout)
    f = forward(theta, X, x_lo, x_hi, nin, H, nout)
    t = (np.asarray(T, np.float64) - y_mean) / y_std
    B = f["Y"].shape[0]
    aY = np.abs(f["Y"] - t) / (B * nout)
    mW3 = aY.T @ np.abs(f["H2"])
    mb3 = aY.sum(0)
    aZ2 = (aY @ np.abs(W3)) * np.abs(silu_grad(f["Z2"]))
    mW2 = aZ2.T @ np.abs(f["H1"])
    mb2 = aZ2.sum(0)
    aZ1 = (aZ2 @ np.abs(W2)) * np.abs(silu_grad(f["Z1"]))
    mW1 = aZ1.T @ np.abs(f["Xn"])
    mb1 = aZ1.sum(0)
    return np.concatenate([mW1.ravel(), mb1, mW2.ravel(), mb2, mW3.ravel(), mb3])
