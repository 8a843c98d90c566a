"""Pins of the reference gradients (oracle.sgemm_backward) by central finite
differences in float64.

L(A, B, C) = sum(G * (alpha*op(A)*op(B) + beta*C)) is linear in every single
entry of A, B and C, so a central difference with step h = 1e-3 equals the
partial derivative up to float64 rounding. This pins the gradient formulas
(and their transposes for all four op combinations) independently of the
library that implements them on the GPU."""
import numpy as np
import pytest

import oracle
import workloads as wl

TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]


def _loss(ta, tb, alpha, A, B, beta, C, G):
    m, n = G.shape
    k = A.shape[1] if ta == "N" else A.shape[0]
    Y = oracle.dgemm(ta, tb, m, n, k, alpha, A, A.shape[0], B, B.shape[0], beta, C, m)
    return float(np.sum(G * Y))


@pytest.mark.parametrize("ta,tb", TRANS)
def test_reference_gradients_match_central_differences(ta, tb):
    m, n, k = 64, 48, 32
    h = 1e-3
    rng = np.random.default_rng(3)
    alpha, beta = 1.25, -0.75
    A = np.asfortranarray(rng.normal(size=wl.stored_shape(ta, m, k)))
    B = np.asfortranarray(rng.normal(size=wl.stored_shape(tb, k, n)))
    C = np.asfortranarray(rng.normal(size=(m, n)))
    G = np.asfortranarray(rng.normal(size=(m, n)))
    dA, dB, dC = oracle.sgemm_backward(ta, tb, alpha, A, B, beta, G)
    assert dA.shape == A.shape and dB.shape == B.shape and dC.shape == C.shape
    for X, dX in ((A, dA), (B, dB), (C, dC)):
        idx = rng.choice(X.size, size=min(X.size, 160), replace=False)
        for flat in idx:
            i, j = np.unravel_index(flat, X.shape)
            x0 = X[i, j]
            X[i, j] = x0 + h
            lp = _loss(ta, tb, alpha, A, B, beta, C, G)
            X[i, j] = x0 - h
            lm = _loss(ta, tb, alpha, A, B, beta, C, G)
            X[i, j] = x0
            fd = (lp - lm) / (2 * h)
            scale = abs(_loss(ta, tb, alpha, A, B, beta, C, G)) + 1.0
            assert abs(fd - dX[i, j]) <= 1e-9 * scale, (ta, tb, i, j, fd, dX[i, j])


def test_reference_gradients_match_torch_float64():
    """Cross-check with an independent library (torch autograd, float64)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    for ta, tb in TRANS:
        m, n, k = 9, 7, 5
        A = rng.normal(size=wl.stored_shape(ta, m, k))
        B = rng.normal(size=wl.stored_shape(tb, k, n))
        G = rng.normal(size=(m, n))
        At = torch.tensor(A, requires_grad=True)
        Bt = torch.tensor(B, requires_grad=True)
        Y = 0.5 * ((At if ta == "N" else At.T) @ (Bt if tb == "N" else Bt.T))
        (Y * torch.tensor(G)).sum().backward()
        dA, dB, _ = oracle.sgemm_backward(ta, tb, 0.5, A, B, 0.0, G)
        assert np.allclose(dA, At.grad.numpy(), rtol=1e-12, atol=1e-12)
        assert np.allclose(dB, Bt.grad.numpy(), rtol=1e-12, atol=1e-12)
