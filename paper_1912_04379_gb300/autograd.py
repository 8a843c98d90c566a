"""Differentiable SGEMM: a torch.autograd.Function whose backward is the
library's gb_sgemm_backward (hand-written gradient products, same kernels).

For C_out = alpha*op(A)*op(B) + beta*C and an upstream gradient G = dL/dC_out:
    dL/dop(A) = alpha * G * op(B)^T,   dL/dop(B) = alpha * op(A)^T * G,
    dL/dC = beta * G,
mapped back through the transposes onto the stored A and B (see
gb_sgemm_backward in include/gbsgemm.h). The paper uses its SGEMM as the
kernel of neural-network training (Sec. 4); `linear` is that dense layer
for row-major torch tensors.
"""
from __future__ import annotations

import torch

from . import api


def _as_colmajor(t):
    """The same values as a column-major (stride(0) == 1) tensor, on the same
    device and in the same dtype; anything but a float32 CUDA tensor is then
    rejected by the SGEMM call (there is no CPU path)."""
    if t.dim() == 2 and (t.stride(0) == 1 or t.shape[0] <= 1) and t.is_cuda and \
            t.dtype == torch.float32:
        return t
    return t.detach().t().contiguous().t()


def _ld(t):
    rows, cols = t.shape
    return max(t.stride(1) if cols > 1 else rows, rows, 1)


class SGEMMFunction(torch.autograd.Function):
    """out = alpha*op(A)*op(B) + beta*C on column-major tensors (C may be None)."""

    @staticmethod
    def forward(ctx, A, B, C, alpha=1.0, beta=0.0, transa="N", transb="N", algo="auto"):
        A = _as_colmajor(A)
        B = _as_colmajor(B)
        m = A.shape[0] if transa in "Nn" else A.shape[1]
        n = B.shape[1] if transb in "Nn" else B.shape[0]
        out = api.colmajor(m, n, device=A.device)
        if C is not None and beta != 0.0:
            out.copy_(C)
        else:
            beta = 0.0
        api.sgemm(A, B, out, alpha=alpha, beta=beta, transa=transa, transb=transb, algo=algo)
        ctx.save_for_backward(A, B)
        ctx.cfg = (alpha, beta, transa, transb, algo, C is not None)
        return out

    @staticmethod
    def backward(ctx, G):
        A, B = ctx.saved_tensors
        alpha, beta, ta, tb, algo, has_c = ctx.cfg
        G = _as_colmajor(G)
        m, n = G.shape
        k = A.shape[1] if ta in "Nn" else A.shape[0]
        need_a, need_b, need_c = ctx.needs_input_grad[:3]
        dA = api.colmajor(*A.shape, device=A.device) if need_a else None
        dB = api.colmajor(*B.shape, device=B.device) if need_b else None
        dC = api.colmajor(m, n, device=G.device) if (need_c and has_c) else None
        api.backward_raw(ta, tb, m, n, k, alpha, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), beta,
                         G.data_ptr(), _ld(G),
                         dA.data_ptr() if dA is not None else 0, _ld(dA) if dA is not None else 1,
                         dB.data_ptr() if dB is not None else 0, _ld(dB) if dB is not None else 1,
                         dC.data_ptr() if dC is not None else 0, _ld(dC) if dC is not None else 1,
                         algo=algo)
        return dA, dB, dC, None, None, None, None, None


def sgemm(A, B, C=None, alpha=1.0, beta=0.0, transa="N", transb="N", algo="auto"):
    """Differentiable out-of-place SGEMM on column-major tensors."""
    return SGEMMFunction.apply(A, B, C, alpha, beta, transa, transb, algo)


def linear(X, W, algo="auto"):
    """Y = X @ W for row-major X (batch x d_in) and W (d_in x d_out).

    Row-major X is the column-major X^T, so Y^T = W^T X^T is one column-major
    SGEMM ('N','N', m = d_out, n = batch, k = d_in) on the same storage.
    """
    Yt = SGEMMFunction.apply(W.t(), X.t(), None, 1.0, 0.0, "N", "N", algo)
    return Yt.t()
