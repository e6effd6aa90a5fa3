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

Pins (tests): gradients against central finite differences; Adam lowers a smooth loss; the
guess vector is a spin singlet of excitation rank <= 2 whose extracted increment is the input;
the feature packing reproduces the space's CAS operator.
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


# ---- the 6e6o space <-> network interface -----------------------------------------------------
#
# Features of a (3,3) space, 708 values: the vacuum-ordered one-body block h[p][q] over the six
# local orbitals (36, row-major), the pair-symmetric two-body block W[p][q][r][s] once per
# unordered pair of index pairs P = 6p+q <= R = 6r+s (666, row-major over (P, R)), and the
# dressed Fock diagonal F_pp of the six orbitals (6).  The space's core energy is left out: a
# constant shift of the CAS operator does not change its eigenvectors.
# Targets, 54 values: the increment X1[i][a] (9, row-major) and X2[i][j][a][b] once per
# unordered pair of (i a), (j b) index pairs, P = 3i+a <= R = 3j+b (45, row-major over (P, R)).

N_FEATURES = 36 + 666 + 6
N_TARGETS = 9 + 45


def _upper_pairs(m: int):
    return [(P, R) for P in range(m) for R in range(P, m)]


def features(e0: float, F: np.ndarray, W: np.ndarray, occ, vir) -> np.ndarray:
    from .cas import space_problem

    _, h, w = space_problem(e0, F, W, occ, vir)
    orb = list(occ) + list(vir)
    wp = w.reshape(36, 36)
    wu = np.array([wp[P, R] for P, R in _upper_pairs(36)])
    return np.concatenate([h.ravel(), wu, np.array([F[o, o] for o in orb])])


def unpack_features(x: np.ndarray):
    """(h[6][6], W[6][6][6][6], F diagonal[6]) from a feature row (inverse of the packing)."""
    h = x[:36].reshape(6, 6)
    wp = np.zeros((36, 36))
    for k, (P, R) in enumerate(_upper_pairs(36)):
        wp[P, R] = wp[R, P] = x[36 + k]
    return h, wp.reshape(6, 6, 6, 6), x[702:708]


def pack_increment(x1: np.ndarray, x2: np.ndarray) -> np.ndarray:
    x2p = x2.transpose(0, 2, 1, 3).reshape(9, 9)   # [3i+a][3j+b]
    return np.concatenate([x1.ravel(), [x2p[P, R] for P, R in _upper_pairs(9)]])


def unpack_increment(y: np.ndarray):
    x1 = y[:9].reshape(3, 3)
    x2p = np.zeros((9, 9))
    for k, (P, R) in enumerate(_upper_pairs(9)):
        x2p[P, R] = x2p[R, P] = y[9 + k]
    return x1, x2p.reshape(3, 3, 3, 3).transpose(0, 2, 1, 3)


def targets(vec: np.ndarray) -> np.ndarray:
    """Packed increment of a (3,3) CI vector with Phi coefficient 1."""
    from .cas import increment

    return pack_increment(*increment(3, 3, vec))


def guess_vector(y: np.ndarray) -> np.ndarray:
    """Start vector of a (3,3) space from a packed increment: the part of e^{X1 + X2} Phi of
    excitation rank <= 2, i.e. Phi + X1 Phi + (X2 + X1^2 / 2) Phi, with X the closed-shell
    cluster operator of the increment (singles sum X1_ia E_ai, doubles half-sum X2_ijab E_ai E_bj)."""
    from .secondq import cas_operators, reference_state

    x1, x2 = unpack_increment(y)
    ops = cas_operators(3, 3)
    phi = np.zeros(ops.basis.dim)
    phi[ops.basis.index(reference_state(6, 3))] = 1.0
    z = np.zeros((3, 3, 3, 3))
    s1 = ops.apply_cluster(x1, z, 3, phi)
    s2 = ops.apply_cluster(np.zeros((3, 3)), x2, 3, phi)
    s11 = ops.apply_cluster(x1, z, 3, s1)
    return phi + s1 + s2 + 0.5 * s11


def column_stats(X: np.ndarray):
    """Mean and population standard deviation of every column (FP64)."""
    mu = X.mean(axis=0)
    sd = np.sqrt(((X - mu) ** 2).mean(axis=0))
    return mu, sd
