"""The product path has no CPU or PyTorch fallback: with the CUDA library
missing it raises, and tensors that are not float32 CUDA tensors are
rejected by the binding instead of being computed some other way."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_missing_library_raises():
    code = ("import paper_1912_04379_gb300.build as b\n"
            "from paper_1912_04379_gb300 import _lib\n"
            "b.LIB = '/nonexistent-dir/libgbsgemm.so'\n"
            "try:\n"
            "    _lib.load(build_if_missing=False)\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "    raise SystemExit(0)\n"
            "raise SystemExit(3)\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "not built" in out.stdout


def test_cpu_tensors_are_rejected():
    torch = pytest.importorskip("torch")
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import autograd
    A = torch.ones((8, 8)).t()                       # column-major, but on the CPU
    B = torch.ones((8, 8)).t()
    C = torch.zeros((8, 8)).t()
    with pytest.raises(TypeError):
        gb.sgemm(A, B, C)
    with pytest.raises(TypeError):
        autograd.sgemm(A, B)
    if torch.cuda.is_available():                    # a GPU run: the dtype check instead
        A64 = torch.ones((8, 8), dtype=torch.float64, device="cuda").t()
        with pytest.raises(TypeError):
            gb.sgemm(A64, A64, A64)
