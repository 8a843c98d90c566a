"""A fully connected network whose forward pass and training step run in the
CUDA library (gb_mlp_forward / gb_mlp_train_step; argument marshalling only).

The paper's application (Sec. 4): the SGEMM as the kernel of neural-network
training. Examples are columns: X is (n_0 x B), Y is (n_L x B); W_l is an
(n_l x n_{l-1}) column-major tensor, b_l has n_l entries, and the layer
outputs H_l and gradients G_l = dE/dZ_l are (n_l x B) column-major tensors
owned by this object. E = sum (H_L - Y)^2 / (2B); hidden layers use tanh (or
the identity), the output layer the identity.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from .api import _stream_ptr, colmajor, default_handle


def _ptrs(ts):
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


class MLP:
    def __init__(self, widths, batch, hidden="tanh", algo="auto", handle=None, device=None):
        if len(widths) < 2:
            raise ValueError("need at least one layer (two widths)")
        self.h = handle or default_handle()
        self.lib = self.h.lib
        self.device = self.h.device if device is None else torch.device(device)
        self.widths = [int(w) for w in widths]
        self.batch = int(batch)
        self.algo = algo
        L = len(widths) - 1
        self._widths_c = (ctypes.c_int64 * (L + 1))(*self.widths)
        self.desc = _lib.MlpDesc(L, self._widths_c, self.batch, _lib.ACTIVATIONS[hidden])
        dev = self.device
        self.W = [colmajor(self.widths[l + 1], self.widths[l], device=dev) for l in range(L)]
        self.b = [torch.zeros(self.widths[l + 1], dtype=torch.float32, device=dev)
                  for l in range(L)]
        self.H = [colmajor(self.widths[l + 1], self.batch, device=dev) for l in range(L)]
        self.G = [colmajor(self.widths[l + 1], self.batch, device=dev) for l in range(L)]
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        nbytes = ctypes.c_size_t(0)
        _lib.check("gb_mlp_workspace_size",
                   self.lib.gb_mlp_workspace_size(_lib.ALGOS[algo], ctypes.byref(self.desc), 1,
                                                  ctypes.byref(nbytes)))
        self.workspace = torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8, device=dev)
        self.ws_bytes = int(nbytes.value)

    @property
    def layers(self):
        return len(self.widths) - 1

    def _check_xy(self, X, rows, name):
        if (X.dtype != torch.float32 or X.device != self.device or tuple(X.shape) !=
                (rows, self.batch) or (rows > 1 and X.stride(0) != 1) or
                (self.batch > 1 and X.stride(1) != rows)):
            raise ValueError(f"{name} must be a dense column-major ({rows} x {self.batch}) "
                             f"float32 tensor on {self.device}")

    def forward(self, X, stream=None):
        """H_1 .. H_L for the input X; returns H_L."""
        self._check_xy(X, self.widths[0], "X")
        _lib.check("gb_mlp_forward", self.lib.gb_mlp_forward(
            self.h.h, _lib.ALGOS[self.algo], ctypes.byref(self.desc), _ptrs(self.W),
            _ptrs(self.b), X.data_ptr(), _ptrs(self.H), self.workspace.data_ptr(),
            self.ws_bytes, _stream_ptr(stream)))
        return self.H[-1]

    def train_step(self, X, Y, lr, stream=None):
        """One gradient-descent step; returns the (device) loss before the update."""
        self._check_xy(X, self.widths[0], "X")
        self._check_xy(Y, self.widths[-1], "Y")
        _lib.check("gb_mlp_train_step", self.lib.gb_mlp_train_step(
            self.h.h, _lib.ALGOS[self.algo], ctypes.byref(self.desc), _ptrs(self.W),
            _ptrs(self.b), X.data_ptr(), Y.data_ptr(), float(lr), _ptrs(self.H), _ptrs(self.G),
            self.loss.data_ptr(), self.workspace.data_ptr(), self.ws_bytes, _stream_ptr(stream)))
        return self.loss
