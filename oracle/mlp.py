"""CPU oracle for one training step of a fully connected network, in double precision.

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`): the tests, the smoke
check and the benchmark's CPU legs use it; the CUDA library neither imports
nor links it.

The paper's application (Sec. 4, last paragraph) is the distributed training
of a large neural network with the SGEMM as the kernel of the training
procedure. This module writes out, from the definitions, the step such a
training procedure takes for a fully connected network with L layers of
widths n_0 .. n_L on a batch of B examples (one example per column):

  forward   Z_l = W_l H_{l-1} + b_l 1^T,  H_l = phi_l(Z_l),  H_0 = X,
            phi_l = tanh (or the identity) for l < L, phi_L = identity;
  loss      E = sum_ij (H_L - Y)_ij^2 / (2B);
  backward  G_L = dE/dZ_L = (H_L - Y) / B,
            G_l = (W_{l+1}^T G_{l+1}) * phi_l'(Z_l)   (elementwise; for tanh
            phi' = 1 - tanh^2 = 1 - H_l^2),
            dE/dW_l = G_l H_{l-1}^T,  dE/db_l = G_l 1;
  update    W_l <- W_l - lr dE/dW_l,  b_l <- b_l - lr dE/db_l (plain gradient
            descent, the update of a data-parallel trainer after its gradients
            are summed).

Matrices are numpy float64 arrays in their mathematical shape (W_l is
n_l x n_{l-1}); the products are numpy matmuls (a library primitive).
"""
from __future__ import annotations

import numpy as np

HIDDEN = ("tanh", "identity")


def _phi(kind, Z):
    """Hidden-layer activation."""
    return np.tanh(Z) if kind == "tanh" else Z.copy()


def _phi_grad_from_output(kind, H):
    """phi'(Z) written through the layer's output H = phi(Z)."""
    return 1.0 - H * H if kind == "tanh" else np.ones_like(H)


def _f64(xs):
    return [np.asarray(x, dtype=np.float64) for x in xs]


def forward(Ws, bs, X, hidden="tanh"):
    """H_1 .. H_L of the forward pass (list of n_l x B arrays)."""
    assert hidden in HIDDEN
    Ws, bs = _f64(Ws), _f64(bs)
    H = np.asarray(X, dtype=np.float64)
    L = len(Ws)
    Hs = []
    for l in range(L):
        Z = Ws[l] @ H + bs[l][:, None]
        H = _phi(hidden, Z) if l < L - 1 else Z
        Hs.append(H)
    return Hs


def loss(Ws, bs, X, Y, hidden="tanh"):
    """E = sum (H_L - Y)^2 / (2B)."""
    HL = forward(Ws, bs, X, hidden)[-1]
    B = HL.shape[1]
    return float(np.sum((HL - np.asarray(Y, dtype=np.float64)) ** 2) / (2 * B))


def grads(Ws, bs, X, Y, hidden="tanh"):
    """(E, Hs, Gs, dWs, dbs): loss, forward outputs, G_l = dE/dZ_l and the
    weight and bias gradients, by the chain rule written above."""
    Ws, bs = _f64(Ws), _f64(bs)
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Hs = forward(Ws, bs, X, hidden)
    L = len(Ws)
    B = X.shape[1]
    R = Hs[-1] - Y
    E = float(np.sum(R * R) / (2 * B))
    Gs = [None] * L
    Gs[L - 1] = R / B
    for l in range(L - 2, -1, -1):
        Gs[l] = (Ws[l + 1].T @ Gs[l + 1]) * _phi_grad_from_output(hidden, Hs[l])
    prev = [X] + Hs[:-1]
    dWs = [Gs[l] @ prev[l].T for l in range(L)]
    dbs = [Gs[l].sum(axis=1) for l in range(L)]
    return E, Hs, Gs, dWs, dbs


def step(Ws, bs, X, Y, lr, hidden="tanh"):
    """One gradient-descent step: (E, Hs, Gs, new Ws, new bs)."""
    E, Hs, Gs, dWs, dbs = grads(Ws, bs, X, Y, hidden)
    Ws, bs = _f64(Ws), _f64(bs)
    newW = [W - lr * dW for W, dW in zip(Ws, dWs)]
    newb = [b - lr * db for b, db in zip(bs, dbs)]
    return E, Hs, Gs, newW, newb
