"""GPU backward: gb_sgemm_backward and the autograd Function against the
FP64 reference gradients (pinned by finite differences on the CPU).

Each gradient is itself an SGEMM (dA reduces over N, dB over M), so the
acceptance per element is the same bound as the forward product with the
gradient's own reduction length and denominator D = |alpha| |G| |op(B)|^T
(resp. |alpha| |op(A)|^T |G|)."""
import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu import STANDARD_BOUND_MIN_K, split_extra, torch_gpu

pytestmark = pytest.mark.gpu
TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]
ALGOS = ("simt", "tf32x3", "bf16x3", "bf16x6", "fp16x3")


def _check(got, want, D, kred, algo, what):
    for extra, must in ((split_extra(algo, kred), True),
                        (0.0, kred >= STANDARD_BOUND_MIN_K[algo])):
        if not must:
            continue
        b = oracle.bound(D, kred, extra)
        ratio = np.abs(got.astype(np.float64) - want) / np.where(b > 0, b, 1.0)
        assert np.all(np.abs(got - want) <= b), f"{what} ({algo}): max ratio {ratio.max()}"


def _abs_grads(ta, tb, alpha, A, B, G):
    """Bound denominators of dA and dB: the same products on |.|."""
    dA, dB, _ = oracle.sgemm_backward(ta, tb, abs(alpha), np.abs(A), np.abs(B), 0.0, np.abs(G))
    return dA, dB


@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("algo", ALGOS)
def test_backward_small_all_transposes(algo, ta, tb):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    m, n, k = 64, 48, 32
    rng = np.random.default_rng(61)
    A = rng.normal(size=wl.stored_shape(ta, m, k)).astype(np.float32)
    B = rng.normal(size=wl.stored_shape(tb, k, n)).astype(np.float32)
    G = rng.normal(size=(m, n)).astype(np.float32)
    alpha, beta = 1.25, -0.75
    cm = lambda x: torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()     # column-major
    dA = gb.colmajor(*A.shape)
    dB = gb.colmajor(*B.shape)
    dC = gb.colmajor(m, n)
    Ad, Bd, Gd = cm(A), cm(B), cm(G)
    gb.backward_raw(ta, tb, m, n, k, alpha, Ad.data_ptr(), A.shape[0], Bd.data_ptr(), B.shape[0],
                    beta, Gd.data_ptr(), m, dA.data_ptr(), A.shape[0], dB.data_ptr(), B.shape[0],
                    dC.data_ptr(), m, algo=algo)
    torch.cuda.synchronize()
    rA, rB, rC = oracle.sgemm_backward(ta, tb, alpha, A, B, beta, G)
    DA, DB = _abs_grads(ta, tb, alpha, A, B, G)
    _check(dA.cpu().numpy(), rA, DA, n, algo, "dA")
    _check(dB.cpu().numpy(), rB, DB, m, algo, "dB")
    assert np.array_equal(dC.cpu().numpy(), (np.float32(beta) * G))


def test_backward_skips_null_outputs():
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    m, n, k = 40, 30, 20
    A = torch.randn(k, m, device="cuda").t()
    B = torch.randn(n, k, device="cuda").t()
    G = torch.randn(n, m, device="cuda").t()
    dB = gb.colmajor(k, n)
    gb.backward_raw("N", "N", m, n, k, 1.0, A.data_ptr(), m, B.data_ptr(), k, 0.0, G.data_ptr(),
                    m, 0, 1, dB.data_ptr(), k, 0, 1, algo="simt")
    torch.cuda.synchronize()
    want = (A.double().t() @ G.double()).float()
    assert torch.allclose(dB, want, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("algo", ("simt", "bf16x6"))
def test_autograd_function_with_c_input(algo):
    torch = torch_gpu()
    from paper_1912_04379_gb300 import autograd as ga
    m, n, k = 70, 50, 40
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn(m, k, device="cuda", generator=g).t().contiguous().t().requires_grad_()
    B = torch.randn(n, k, device="cuda", generator=g).t().contiguous().t().requires_grad_()
    C = torch.randn(n, m, device="cuda", generator=g).t().requires_grad_()
    Gup = torch.randn(m, n, device="cuda", generator=g)
    out = ga.sgemm(A, B, C, alpha=0.5, beta=2.0, transa="N", transb="T", algo=algo)
    (out * Gup).sum().backward()
    rA, rB, rC = oracle.sgemm_backward("N", "T", 0.5, A.detach().cpu().numpy(),
                                       B.detach().cpu().numpy(), 2.0, Gup.cpu().numpy())
    DA, DB = _abs_grads("N", "T", 0.5, A.detach().cpu().numpy(), B.detach().cpu().numpy(),
                        Gup.cpu().numpy())
    _check(A.grad.cpu().numpy(), rA, DA, n, algo, "dA")
    _check(B.grad.cpu().numpy(), rB, DB, m, algo, "dB")
    assert np.array_equal(C.grad.cpu().numpy(), 2.0 * Gup.cpu().numpy())


def test_dense_layer_4096x1024x4096():
    """Y = X W (X 4096 x 1024, W 1024 x 4096 ~ N(0, 1/1024)), loss = sum(Y * G):
    forward and both gradients on sampled columns against the oracle."""
    torch = torch_gpu()
    from paper_1912_04379_gb300 import autograd as ga
    X, W, G = wl.dense_layer()
    Xd = torch.from_numpy(X).cuda().requires_grad_()
    Wd = torch.from_numpy(W).cuda().requires_grad_()
    Gd = torch.from_numpy(G).cuda()
    Y = ga.linear(Xd, Wd, algo="auto")
    (Y * Gd).sum().backward()
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    # forward: Y^T = W^T X^T (column-major, m = 4096, n = 4096, k = 1024); column j of Y^T = row j of Y
    cols = np.unique(rng.integers(0, 4096, 6))
    Wt = np.asfortranarray(W.T)          # column-major view of row-major W storage
    Xt = np.asfortranarray(X.T)
    C64, D = oracle.sgemm("N", "N", 4096, 4096, 1024, 1.0, Wt, 4096, Xt, 1024, 0.0, None, 4096,
                          cols=cols)
    got = Y.detach().cpu().numpy()[cols, :].T
    assert oracle.err_report(got, C64, D, 1024)["max_ratio"] <= 1.0
    # dX = G W^T (4096 x 1024): rows of dX are columns of dX^T = W G^T
    Gt = np.asfortranarray(G.T)
    rows = np.unique(rng.integers(0, 4096, 6))
    R64, RD = oracle.sgemm("N", "N", 1024, 4096, 4096, 1.0, np.asfortranarray(W), 1024, Gt, 4096,
                           0.0, None, 1024, cols=rows)
    gotx = Xd.grad.cpu().numpy()[rows, :].T
    assert oracle.err_report(gotx, R64, RD, 4096)["max_ratio"] <= 1.0
    # dW = X^T G (1024 x 4096): rows of dW are columns of dW^T = G^T X
    wrows = np.unique(rng.integers(0, 1024, 6))
    S64, SD = oracle.sgemm("N", "N", 4096, 1024, 4096, 1.0, Gt, 4096, np.asfortranarray(X), 4096,
                           0.0, None, 4096, cols=wrows)
    gotw = Wd.grad.cpu().numpy()[wrows, :].T
    assert oracle.err_report(gotw, S64, SD, 4096)["max_ratio"] <= 1.0
