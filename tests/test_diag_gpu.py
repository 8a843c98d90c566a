"""The FP32 FMA measurement aid: runs, reports the FMA count of its launch,
and measures a rate between a tenth of and about the nominal FP32 peak."""
import ctypes

import pytest

from _gpu import torch_gpu

pytestmark = pytest.mark.gpu


def test_measure_ffma():
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    h = gb.default_handle()
    sink = torch.empty(256, device="cuda")
    fmas = ctypes.c_int64(0)
    s = torch.cuda.current_stream()
    assert h.lib.gb_measure_ffma(h.h, 0, sink.data_ptr(), ctypes.byref(fmas), None) == _lib.GB_ERR_ARG
    assert h.lib.gb_measure_ffma(h.h, 256, sink.data_ptr(), ctypes.byref(fmas), None) == 0
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    assert h.lib.gb_measure_ffma(h.h, 2048, sink.data_ptr(), ctypes.byref(fmas),
                                 ctypes.c_void_p(s.cuda_stream)) == 0
    e1.record(s)
    torch.cuda.synchronize()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert fmas.value == sms * 8 * 256 * 2048 * 16 * 8
    tflops = 2.0 * fmas.value / (e0.elapsed_time(e1) * 1e-3) / 1e12
    nominal = sms * 128 * 2 * 2.1e9 / 1e12
    assert 0.1 * nominal < tflops < 1.05 * nominal, (tflops, nominal)
