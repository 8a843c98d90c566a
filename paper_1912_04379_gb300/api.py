"""Python binding of the C ABI over torch CUDA tensors (marshalling only).

A column-major matrix is a 2-D float32 CUDA tensor whose first stride is 1
(element (r, c) at offset r + c*ld, ld = stride(1)); `colmajor(rows, cols)`
makes one. A row-major torch matrix X (rows x cols, contiguous) is the
column-major matrix X^T, which is how `linear` maps a dense layer onto the
BLAS call. Every computation runs in the CUDA library; nothing here falls
back to torch arithmetic.
"""
from __future__ import annotations

import ctypes
import threading

import torch

from . import _lib

_tls = threading.local()


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def colmajor(rows: int, cols: int, ld: int | None = None, device="cuda", fill=None):
    """A (rows x cols) column-major float32 tensor with leading dimension ld."""
    ld = max(rows, 1) if ld is None else ld
    if ld < max(rows, 1):
        raise ValueError("ld < rows")
    store = torch.empty((max(cols, 1), ld), dtype=torch.float32, device=device)
    if fill is not None:
        store.fill_(fill)
    return store.t()[:rows, :cols]


def from_fortran(arr, device="cuda", rows=None):
    """Upload a Fortran-ordered numpy (ld, cols) float32 array; returns the
    padded storage view (ld x cols) and the logical (rows x cols) view."""
    import numpy as np
    a = np.asarray(arr)
    if a.dtype != np.float32 or not a.flags.f_contiguous:
        raise TypeError("expected a Fortran-ordered float32 array")
    ld, cols = a.shape
    store = torch.from_numpy(np.ascontiguousarray(a.T)).to(device)      # (cols, ld) row-major
    full = store.t()
    return full, full[: (ld if rows is None else rows), :]


def to_fortran(t):
    """Download a column-major tensor view into a Fortran numpy array."""
    return t.detach().t().contiguous().cpu().numpy().T


def _mat(t, name):
    if t is None:
        return 0, 0, 0, 1
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda or t.dim() != 2:
        raise TypeError(f"{name} must be a 2-D float32 CUDA tensor")
    rows, cols = t.shape
    if rows > 1 and cols > 0 and t.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    ld = t.stride(1) if cols > 1 else max(rows, 1)
    ld = max(ld, rows, 1)
    return t.data_ptr(), rows, cols, ld


class Handle:
    """Owns a gb_handle_t bound to one CUDA device and a cached workspace."""

    def __init__(self, device=None):
        self.lib = _lib.load()
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else
                           torch.device(device).index or 0)
        self.device = dev
        with torch.cuda.device(dev):
            h = ctypes.c_void_p()
            _lib.check("gb_create", self.lib.gb_create(ctypes.byref(h)))
        self.h = h
        self._ws = None

    def close(self):
        if self.h is not None and self.h.value:
            self.lib.gb_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace(self, nbytes: int):
        if nbytes == 0:
            return None
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        return self._ws

    def set_fused_split(self, enable: bool):
        """Allow or forbid (default) the split fused into the tensor-core kernel."""
        _lib.check("gb_set_fused_split", self.lib.gb_set_fused_split(self.h, 1 if enable else 0))

    def set_skinny_split(self, enable: bool):
        """Allow (default) or forbid the skinny-product kernel (one side <= 64 rows)."""
        _lib.check("gb_set_skinny_split", self.lib.gb_set_skinny_split(self.h, 1 if enable else 0))

    def skinny_split(self) -> bool:
        v = ctypes.c_int(0)
        _lib.check("gb_get_skinny_split", self.lib.gb_get_skinny_split(self.h, ctypes.byref(v)))
        return bool(v.value)

    def set_promotion(self, k_chunk: int):
        """Promoted accumulation: a fresh tensor-core accumulator every k_chunk
        elements of K, chunks added in FP32 round-to-nearest (0 = off)."""
        _lib.check("gb_set_promotion", self.lib.gb_set_promotion(self.h, int(k_chunk)))

    def promotion(self) -> int:
        v = ctypes.c_int64(0)
        _lib.check("gb_get_promotion", self.lib.gb_get_promotion(self.h, ctypes.byref(v)))
        return v.value

    def tune_grouped(self):
        """Run the grouped autotuner now (synchronises)."""
        _lib.check("gb_tune_grouped", self.lib.gb_tune_grouped(self.h))

    def tune_sgemm(self, algo, transa, transb, m, n, k):
        """Measure the tensor-core row width for this shape bucket (synchronises)."""
        _lib.check("gb_tune_sgemm", self.lib.gb_tune_sgemm(
            self.h, _lib.ALGOS[algo], transa.encode(), transb.encode(), m, n, k))

    def tuning(self):
        """The handle's tuning record (a ctypes gb_tuning_t)."""
        t = _lib.Tuning()
        _lib.check("gb_get_tuning", self.lib.gb_get_tuning(self.h, ctypes.byref(t)))
        return t

    def set_tuning(self, t):
        _lib.check("gb_set_tuning", self.lib.gb_set_tuning(self.h, ctypes.byref(t)))

    def set_wait_limit(self, microseconds: int):
        _lib.check("gb_set_wait_limit", self.lib.gb_set_wait_limit(self.h, int(microseconds)))

    def device_error(self, stream=None):
        """Returns (status, site); status GB_ERR_TIMEOUT if a bounded wait expired."""
        site = ctypes.c_int(0)
        rc = self.lib.gb_get_device_error(self.h, _stream_ptr(stream), ctypes.byref(site))
        return rc, site.value


def default_handle() -> Handle:
    dev = torch.cuda.current_device()
    hs = getattr(_tls, "handles", None)
    if hs is None:
        hs = _tls.handles = {}
    if dev not in hs:
        hs[dev] = Handle(dev)
    return hs[dev]


def workspace_size(algo, transa, transb, m, n, k) -> int:
    lib = _lib.load()
    out = ctypes.c_size_t(0)
    _lib.check("gb_sgemm_workspace_size",
               lib.gb_sgemm_workspace_size(_lib.ALGOS[algo], transa.encode(), transb.encode(),
                                           m, n, k, ctypes.byref(out)))
    return out.value


def sgemm_raw(transa, transb, m, n, k, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc,
              algo="auto", handle=None, stream=None, workspace=None, check=True) -> int:
    """Direct call of gb_sgemm on device pointers (ints). Returns the status."""
    h = handle or default_handle()
    ws_bytes = workspace_size(algo, transa, transb, m, n, k) if (m >= 0 and n >= 0 and k >= 0
                                                                   and transa in "NnTtCc"
                                                                   and transb in "NnTtCc") else 0
    ws = workspace if workspace is not None else h.workspace(ws_bytes)
    ws_ptr = ws.data_ptr() if ws is not None else 0
    ws_len = ws.numel() if ws is not None else 0
    rc = h.lib.gb_sgemm(h.h, _lib.ALGOS[algo], transa.encode(), transb.encode(), m, n, k,
                        float(alpha), A_ptr, lda, B_ptr, ldb, float(beta), C_ptr, ldc,
                        ws_ptr, ws_len, _stream_ptr(stream))
    if check:
        _lib.check("gb_sgemm", rc)
    return rc


def sgemm_host_workspace_size(algo, transa, transb, m, n, k) -> int:
    lib = _lib.load()
    out = ctypes.c_size_t(0)
    _lib.check("gb_sgemm_host_workspace_size",
               lib.gb_sgemm_host_workspace_size(_lib.ALGOS[algo], transa.encode(),
                                                transb.encode(), m, n, k, ctypes.byref(out)))
    return out.value


def sgemm_host_raw(transa, transb, m, n, k, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc,
                   algo="auto", handle=None, stream=None, workspace=None, check=True) -> int:
    """gb_sgemm_host: A, B, C are HOST pointers (ints; page-locked memory for
    overlap), the workspace is device memory. Returns the status."""
    h = handle or default_handle()
    if workspace is None:
        ok = (m >= 0 and n >= 0 and k >= 0 and transa in "NnTtCc" and transb in "NnTtCc")
        workspace = h.workspace(sgemm_host_workspace_size(algo, transa, transb, m, n, k)
                                if ok else 0)
    ws_ptr = workspace.data_ptr() if workspace is not None else 0
    ws_len = workspace.numel() if workspace is not None else 0
    rc = h.lib.gb_sgemm_host(h.h, _lib.ALGOS[algo], transa.encode(), transb.encode(), m, n, k,
                             float(alpha), A_ptr, lda, B_ptr, ldb, float(beta), C_ptr, ldc,
                             ws_ptr, ws_len, _stream_ptr(stream))
    if check:
        _lib.check("gb_sgemm_host", rc)
    return rc


def ssyrk_raw(uplo, trans, n, k, alpha, A_ptr, lda, beta, C_ptr, ldc, algo="auto",
              handle=None, stream=None, check=True) -> int:
    """gb_ssyrk on device pointers: C <- alpha op(A) op(A)^T + beta C on the
    `uplo` triangle. Returns the status."""
    h = handle or default_handle()
    need = ctypes.c_size_t(0)
    rc = h.lib.gb_ssyrk_workspace_size(_lib.ALGOS[algo], uplo.encode(), trans.encode(), n, k,
                                       ctypes.byref(need))
    ws = h.workspace(need.value) if rc == 0 else None
    rc = h.lib.gb_ssyrk(h.h, _lib.ALGOS[algo], uplo.encode(), trans.encode(), n, k, float(alpha),
                        A_ptr, lda, float(beta), C_ptr, ldc, ws.data_ptr() if ws is not None else 0,
                        ws.numel() if ws is not None else 0, _stream_ptr(stream))
    if check:
        _lib.check("gb_ssyrk", rc)
    return rc


def strsm_raw(side, uplo, transa, diag, m, n, alpha, A_ptr, lda, B_ptr, ldb, algo="auto",
              handle=None, stream=None, check=True) -> int:
    """gb_strsm on device pointers: B <- X with op(A) X = alpha B (side 'L') or
    X op(A) = alpha B (side 'R'). Returns the status."""
    h = handle or default_handle()
    need = ctypes.c_size_t(0)
    rc = h.lib.gb_strsm_workspace_size(_lib.ALGOS[algo], side.encode(), uplo.encode(),
                                       transa.encode(), diag.encode(), m, n, ctypes.byref(need))
    ws = h.workspace(need.value) if rc == 0 else None
    rc = h.lib.gb_strsm(h.h, _lib.ALGOS[algo], side.encode(), uplo.encode(), transa.encode(),
                        diag.encode(), m, n, float(alpha), A_ptr, lda, B_ptr, ldb,
                        ws.data_ptr() if ws is not None else 0,
                        ws.numel() if ws is not None else 0, _stream_ptr(stream))
    if check:
        _lib.check("gb_strsm", rc)
    return rc


def pack_size(algo, which, mn, k) -> int:
    lib = _lib.load()
    out = ctypes.c_size_t(0)
    _lib.check("gb_sgemm_pack_size",
               lib.gb_sgemm_pack_size(_lib.ALGOS[algo], which.encode(), mn, k, ctypes.byref(out)))
    return out.value


def pack_raw(algo, which, trans, mn, k, X_ptr, ldx, packed, handle=None, stream=None,
             check=True) -> int:
    """Split and pack op(A) (which='A', mn=M) or op(B) (which='B', mn=N) into
    the uint8 CUDA tensor `packed`."""
    h = handle or default_handle()
    rc = h.lib.gb_sgemm_pack(h.h, _lib.ALGOS[algo], which.encode(), trans.encode(), mn, k,
                             X_ptr, ldx, packed.data_ptr(), packed.numel(), _stream_ptr(stream))
    if check:
        _lib.check("gb_sgemm_pack", rc)
    return rc


def compute_raw(algo, m, n, k, alpha, Apacked, Bpacked, beta, C_ptr, ldc, handle=None,
                stream=None, check=True) -> int:
    """C <- alpha*op(A)*op(B) + beta*C from packed operands."""
    h = handle or default_handle()
    rc = h.lib.gb_sgemm_compute(h.h, _lib.ALGOS[algo], m, n, k, float(alpha),
                                Apacked.data_ptr(), Bpacked.data_ptr(), float(beta), C_ptr, ldc,
                                _stream_ptr(stream))
    if check:
        _lib.check("gb_sgemm_compute", rc)
    return rc


def sgemm(A, B, C, alpha=1.0, beta=0.0, transa="N", transb="N", algo="auto", handle=None,
          stream=None):
    """C <- alpha*op(A)*op(B) + beta*C in place on column-major tensors."""
    pa, ar, ac, lda = _mat(A, "A")
    pb, br, bc, ldb = _mat(B, "B")
    pc, m, n, ldc = _mat(C, "C")
    k = ac if transa in "Nn" else ar
    if (ar if transa in "Nn" else ac) != m or (bc if transb in "Nn" else br) != n or \
            (br if transb in "Nn" else bc) != k:
        raise ValueError("inconsistent shapes for sgemm")
    sgemm_raw(transa, transb, m, n, k, alpha, pa, lda, pb, ldb, beta, pc, ldc, algo=algo,
              handle=handle, stream=stream)
    return C


def backward_raw(transa, transb, m, n, k, alpha, A_ptr, lda, B_ptr, ldb, beta, dC_ptr, lddc,
                 dA_ptr, ldda, dB_ptr, lddb, dCin_ptr, lddcin, algo="auto", handle=None,
                 stream=None, check=True) -> int:
    h = handle or default_handle()
    out = ctypes.c_size_t(0)
    rc = h.lib.gb_sgemm_backward_workspace_size(_lib.ALGOS[algo], transa.encode(),
                                                transb.encode(), m, n, k, ctypes.byref(out))
    if rc != 0:
        if check:
            _lib.check("gb_sgemm_backward_workspace_size", rc)
        return rc
    ws = h.workspace(out.value)
    rc = h.lib.gb_sgemm_backward(h.h, _lib.ALGOS[algo], transa.encode(), transb.encode(), m, n, k,
                                 float(alpha), A_ptr, lda, B_ptr, ldb, float(beta), dC_ptr, lddc,
                                 dA_ptr, ldda, dB_ptr, lddb, dCin_ptr, lddcin,
                                 ws.data_ptr() if ws is not None else 0,
                                 ws.numel() if ws is not None else 0, _stream_ptr(stream))
    if check:
        _lib.check("gb_sgemm_backward", rc)
    return rc


def upload_problems(problems, device="cuda"):
    """Copy host problems (objects with ta, tb, m, n, k, alpha, beta and
    Fortran float32 arrays A, B, C with lda, ldb, ldc) into one device buffer.

    Returns (buffer, tuples, c_views): `tuples` are GroupedPlan problem tuples
    with device pointers; c_views[i] is the (ldc x n) storage view of C_i.
    Each matrix starts on a 256-byte boundary of the buffer.
    """
    import numpy as np
    sizes, offs, off = [], [], 0
    for p in problems:
        for X in (p.A, p.B, p.C):
            offs.append(off)
            sizes.append(X.size)
            off += (X.size + 63) // 64 * 64
    host = np.zeros(max(off, 1), dtype=np.float32)
    i = 0
    for p in problems:
        for X in (p.A, p.B, p.C):
            host[offs[i]:offs[i] + X.size] = X.ravel(order="F")
            i += 1
    buf = torch.from_numpy(host).to(device)
    base = buf.data_ptr()
    tuples, views = [], []
    for j, p in enumerate(problems):
        oa, ob, oc = offs[3 * j:3 * j + 3]
        tuples.append((p.ta, p.tb, p.m, p.n, p.k, p.alpha, p.beta, base + 4 * oa, p.lda,
                       base + 4 * ob, p.ldb, base + 4 * oc, p.ldc))
        ldc, cols = p.C.shape
        views.append(buf[oc:oc + ldc * cols].view(cols, ldc).t())
    return buf, tuples, views


class GroupedPlan:
    """A planned batch of independent SGEMMs for one persistent launch.

    `problems` is a sequence of (transa, transb, m, n, k, alpha, beta, A_ptr,
    lda, B_ptr, ldb, C_ptr, ldc) with device pointers as ints. `run()` only
    enqueues work (graph-capturable); the plan owns its device tables until
    `close()`.
    """

    def __init__(self, problems, algo="auto", handle=None):
        self.h = handle or default_handle()
        lib = self.h.lib
        n = len(problems)
        arr = (_lib.GemmProblem * max(n, 1))()
        for i, (ta, tb, m, nn, k, alpha, beta, A, lda, B, ldb, C, ldc) in enumerate(problems):
            arr[i] = _lib.GemmProblem(ta.encode(), tb.encode(), m, nn, k, float(alpha),
                                      float(beta), A, lda, B, ldb, C, ldc)
        plan = ctypes.c_void_p()
        ws = ctypes.c_size_t(0)
        bad = ctypes.c_int64(-1)
        rc = lib.gb_sgemm_grouped_plan(self.h.h, _lib.ALGOS[algo], n, arr, ctypes.byref(plan),
                                       ctypes.byref(ws), ctypes.byref(bad))
        self.bad_index = bad.value
        if rc != 0:
            err = _lib.GBError("gb_sgemm_grouped_plan", rc)
            err.bad_index = bad.value
            raise err
        self.plan = plan
        self.ws_bytes = ws.value
        self.workspace = torch.empty(max(int(ws.value), 256), dtype=torch.uint8,
                                     device=self.h.device)

    def run(self, stream=None, check=True) -> int:
        rc = self.h.lib.gb_sgemm_grouped_run(self.plan, self.workspace.data_ptr(),
                                             self.workspace.numel(), _stream_ptr(stream))
        if check:
            _lib.check("gb_sgemm_grouped_run", rc)
        return rc

    def close(self):
        if getattr(self, "plan", None) is not None and self.plan.value:
            self.h.lib.gb_sgemm_grouped_destroy(self.plan)
            self.plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def err_report(C, C64, D, k, handle=None, stream=None) -> dict:
    """GPU error report of an FP32 result against FP64 (C64, D) (column-major tensors)."""
    h = handle or default_handle()
    pc, m, n, ldc = _mat(C, "C")
    for t, nm in ((C64, "C64"), (D, "D")):
        if t.dtype != torch.float64 or not t.is_cuda or t.shape != (m, n) or (m > 1 and t.stride(0) != 1):
            raise TypeError(f"{nm} must be a column-major float64 CUDA tensor of shape {(m, n)}")
    ld64 = max(C64.stride(1) if n > 1 else m, m, 1)
    ldd = max(D.stride(1) if n > 1 else m, m, 1)
    need = h.lib.gb_err_report_workspace_size(m, n)
    ws = torch.empty(max(int(need), 1), dtype=torch.uint8, device=h.device)
    rep = _lib.ErrReport()
    _lib.check("gb_err_report",
               h.lib.gb_err_report(h.h, m, n, k, pc, ldc, C64.data_ptr(), ld64, D.data_ptr(), ldd,
                                   ws.data_ptr(), ws.numel(), ctypes.byref(rep),
                                   _stream_ptr(stream)))
    num = rep.sum_sq_diff ** 0.5
    den = rep.sum_sq_ref ** 0.5
    normwise = 0.0 if num == 0.0 else (num / den if den > 0 else float("inf"))
    return dict(max_ratio=rep.max_ratio, median_ratio=rep.median_ratio, normwise=normwise,
                n_fail=rep.n_fail, count=rep.count, sum_sq_diff=rep.sum_sq_diff,
                sum_sq_ref=rep.sum_sq_ref)
