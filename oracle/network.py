"""CPU reference of the learned preconditioner network (test infrastructure
only): a two-layer 1-D convolutional network over the cells of a slab,

  h1[p, j, o] = tanh(b1[o] + sum_{c, d} W1[o, c, d] x[p, j + d - 2, c])
  y[p, j, a]  = b2[a] + sum_{o, d} W2[a, o, d] h1[p, j + d - 2, o]
  loss        = mean over (p, j, a) of (y - t)^2

with zero padding outside the cells, d = 0..4, 26 input channels (13
moments -- {1, v, |v|^2}, the traceless stress and the heat flux -- of a
Krylov vector and of its upwind sweep) and 5 outputs (the coefficients of the macroscopic correction
M_j (c0 + c.v + c4 |v|^2)).  The network has no counterpart in the paper;
it stands in for the synthetic acceleration the paper points to (Sec. 5.2).
Parameters are packed as [W1 (H,26,5), b1 (H), W2 (5,H,5), b2 (5)].
FP64, plain loops over the kernel taps.
"""
import numpy as np

C_IN, C_OUT, WIDTH = 26, 5, 5


def param_count(hidden):
    return hidden * C_IN * WIDTH + hidden + C_OUT * hidden * WIDTH + C_OUT


def unpack(theta, hidden):
    i = 0
    W1 = theta[i:i + hidden * C_IN * WIDTH].reshape(hidden, C_IN, WIDTH)
    i += hidden * C_IN * WIDTH
    b1 = theta[i:i + hidden]
    i += hidden
    W2 = theta[i:i + C_OUT * hidden * WIDTH].reshape(C_OUT, hidden, WIDTH)
    i += C_OUT * hidden * WIDTH
    b2 = theta[i:i + C_OUT]
    return W1, b1, W2, b2


def _shift(a, d):
    """a[:, j + d] with zeros outside (a: (P, nx, C))."""
    out = np.zeros_like(a)
    nx = a.shape[1]
    if d >= 0:
        out[:, :nx - d] = a[:, d:]
    else:
        out[:, -d:] = a[:, :nx + d]
    return out


def forward(theta, hidden, x):
    W1, b1, W2, b2 = unpack(theta, hidden)
    z1 = np.broadcast_to(b1, x.shape[:2] + (hidden,)).copy()
    for d in range(WIDTH):
        z1 += _shift(x, d - 2) @ W1[:, :, d].T
    h1 = np.tanh(z1)
    y = np.broadcast_to(b2, x.shape[:2] + (C_OUT,)).copy()
    for d in range(WIDTH):
        y += _shift(h1, d - 2) @ W2[:, :, d].T
    return y, h1


def loss_and_grad(theta, hidden, x, t):
    """Mean squared error and its gradient (backpropagation, FP64)."""
    W1, b1, W2, b2 = unpack(theta, hidden)
    y, h1 = forward(theta, hidden, x)
    n = y.size
    loss = ((y - t) ** 2).sum() / n
    dy = 2.0 * (y - t) / n
    gW2 = np.zeros_like(W2)
    for d in range(WIDTH):
        sh = _shift(h1, d - 2)
        gW2[:, :, d] = np.einsum("pja,pjo->ao", dy, sh)
    gb2 = dy.sum(axis=(0, 1))
    dh1 = np.zeros_like(h1)
    for d in range(WIDTH):
        # y[j] uses h1[j + d - 2]: gradient flows back to h1[j'] from y[j' - d + 2]
        dh1 += _shift(dy, -(d - 2)) @ W2[:, :, d]
    dz1 = dh1 * (1.0 - h1 * h1)
    gW1 = np.zeros_like(W1)
    for d in range(WIDTH):
        sx = _shift(x, d - 2)
        gW1[:, :, d] = np.einsum("pjo,pjc->oc", dz1, sx)
    gb1 = dz1.sum(axis=(0, 1))
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2])
    return loss, grad
