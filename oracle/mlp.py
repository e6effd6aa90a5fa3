"""FP64 reference of the warm-start network (forward, backward, Adam step).

Not in the paper: the flow can start each space's Davidson solver from a network's guess of
the space's increment instead of Phi.  The network maps a space's dressed-integral features
to its converged increment (X1 and the symmetric part of X2); the plain solver stays the
judge, so energies do not depend on it.  This module is the FP64 definition the GPU kernels
are checked against.

Network: two hidden tanh layers,
    H1 = tanh(X W1 + b1),  H2 = tanh(H1 W2 + b2),  Y = H2 W3 + b3,
loss L = 1/(2N) sum_n sum_o (Y - T)^2.  Parameters are packed as [W1, b1, W2, b2, W3, b3] with
W stored [fan_in][fan_out] row-major.  Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Pins: gradients against central finite differences (tests).
"""
from __future__ import annotations

import numpy as np


def shapes(n_in: int, n_hidden: int, n_out: int):
    return [(n_in, n_hidden), (n_hidden,), (n_hidden, n_hidden), (n_hidden,), (n_hidden, n_out), (n_out,)]


def param_count(n_in: int, n_hidden: int, n_out: int) -> int:
    return sum(int(np.prod(s)) for s in shapes(n_in, n_hidden, n_out))


def unpack(p: np.ndarray, n_in: int, n_hidden: int, n_out: int):
    out, off = [], 0
    for s in shapes(n_in, n_hidden, n_out):
        k = int(np.prod(s))
        out.append(p[off:off + k].reshape(s))
        off += k
    return out


def init_params(n_in: int, n_hidden: int, n_out: int, seed: int) -> np.ndarray:
    """Seeded Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in shapes(n_in, n_hidden, n_out):
        if len(s) == 2:
            lim = np.sqrt(6.0 / (s[0] + s[1]))
            parts.append(rng.uniform(-lim, lim, size=s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)


def forward(p, X, n_in, n_hidden, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, n_hidden, n_out)
    H1 = np.tanh(X @ W1 + b1)
    H2 = np.tanh(H1 @ W2 + b2)
    return H2 @ W3 + b3, (H1, H2)


def loss_and_grad(p, X, T, n_in, n_hidden, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, n_hidden, n_out)
    N = X.shape[0]
    Y, (H1, H2) = forward(p, X, n_in, n_hidden, n_out)
    R = Y - T
    L = 0.5 * float(np.sum(R * R)) / N
    dY = R / N
    gW3 = H2.T @ dY
    gb3 = dY.sum(axis=0)
    dZ2 = (dY @ W3.T) * (1.0 - H2 * H2)
    gW2 = H1.T @ dZ2
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2.T) * (1.0 - H1 * H1)
    gW1 = X.T @ dZ1
    gb1 = dZ1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def adam_step(p, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
