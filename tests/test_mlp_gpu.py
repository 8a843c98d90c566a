"""GPU parity of the training step (gb_mlp_forward / gb_mlp_train_step) against
the FP64 oracle, stage by stage.

Each stage is checked with the GPU's own inputs to that stage (the previous
layer's output, the incoming gradient), so every check is one GEMM bound plus
a few roundings, derived per stage:

  forward   h = phi(fl(Z + b)), Z the GEMM: |h - phi(Z64 + b)| <= eZ (1 + u)
            + u |Z64 + b| + (tanh only) 2 ulp(h) for CUDA's tanhf;
  loss grad G_L = fl(fl(H - Y) / B): |G - (H - Y)/B| <= (2u + u^2) |H - Y| / B;
  loss      (N + 4) u E for the fixed-order sum of N squares;
  backward  G = fl(P * fl(1 - h^2)), P the GEMM: |G - P64 (1 - h^2)|
            <= (eP (1 + u)^2 + (2u + u^2) |P64|) |1 - h^2|;
  update    W' is one GEMM (alpha = -lr, beta = 1): its own bound;
  bias      b' = fma(-lr, s, b), s the row sum in any order:
            |b' - (b - lr sum G)| <= |lr| B u sum|G| + u |b'|.

eZ, eP are the per-element GEMM bounds (2 max(K,1) u + e_algo) D of the
algorithm that ran.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from _gpu import auto_algo, split_extra, torch_gpu

pytestmark = pytest.mark.gpu
U = 2.0 ** -24
TINY = 2.0 ** -126


def _resolve(algo, k):
    if algo != "auto":
        return algo
    return auto_algo(k)


def _gemm_bound(algo, k, D):
    a = _resolve(algo, k)
    return (2 * max(k, 1) * U + split_extra(a, k)) * D


def _setup(widths, batch, hidden, algo, seed):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    rng = np.random.default_rng(seed)
    L = len(widths) - 1
    Ws = [rng.normal(0, 1 / np.sqrt(widths[l]), (widths[l + 1], widths[l])).astype(np.float32)
          for l in range(L)]
    bs = [rng.normal(0, 0.1, widths[l + 1]).astype(np.float32) for l in range(L)]
    X = rng.normal(0, 1, (widths[0], batch)).astype(np.float32)
    Y = rng.normal(0, 1, (widths[-1], batch)).astype(np.float32)
    net = gb.MLP(widths, batch, hidden=hidden, algo=algo)
    for l in range(L):
        net.W[l].copy_(torch.from_numpy(Ws[l]))
        net.b[l].copy_(torch.from_numpy(bs[l]))
    Xd = gb.colmajor(widths[0], batch)
    Xd.copy_(torch.from_numpy(X))
    Yd = gb.colmajor(widths[-1], batch)
    Yd.copy_(torch.from_numpy(Y))
    return net, Ws, bs, X, Y, Xd, Yd


def _np(t):
    return t.detach().cpu().numpy().astype(np.float32)


def _gemm64(ta, tb, alpha, A, B, beta=0.0, C=None):
    """Oracle GEMM on mathematical-shape float32 arrays: (C64, D)."""
    A = np.asfortranarray(A, dtype=np.float32)
    B = np.asfortranarray(B, dtype=np.float32)
    m = A.shape[1] if ta == "T" else A.shape[0]
    k = A.shape[0] if ta == "T" else A.shape[1]
    n = B.shape[0] if tb == "T" else B.shape[1]
    Cf = None if C is None else np.asfortranarray(C, dtype=np.float32)
    return oracle.sgemm(ta, tb, m, n, k, alpha, A, A.shape[0], B, B.shape[0], beta,
                        Cf, m if Cf is not None else m)


def _check_forward(net, Ws, bs, X, hidden, algo):
    L = len(Ws)
    prev = X
    for l in range(L):
        Z64, D = _gemm64("N", "N", 1.0, Ws[l], prev)
        eZ = _gemm_bound(algo, Ws[l].shape[1], D)
        pre = Z64 + bs[l].astype(np.float64)[:, None]
        H = _np(net.H[l]).astype(np.float64)
        tanh_layer = hidden == "tanh" and l < L - 1
        want = np.tanh(pre) if tanh_layer else pre
        tol = eZ * (1 + U) + U * np.abs(pre) + TINY
        if tanh_layer:
            tol = tol + 2 * 2.0 ** -23 * np.maximum(np.abs(want), np.abs(H))
        bad = np.abs(H - want) > tol
        assert not bad.any(), (l, int(bad.sum()), float(np.max(np.abs(H - want) / tol)))
        prev = _np(net.H[l])


@pytest.mark.parametrize("hidden", ("tanh", "identity"))
@pytest.mark.parametrize("algo", ("simt", "bf16x6", "auto"))
def test_forward_layerwise(hidden, algo):
    torch = torch_gpu()
    widths, batch = (96, 130, 70, 10), 77
    net, Ws, bs, X, Y, Xd, Yd = _setup(widths, batch, hidden, algo, seed=50)
    net.forward(Xd)
    torch.cuda.synchronize()
    _check_forward(net, Ws, bs, X, hidden, algo)


CASES = [((96, 130, 70, 10), 77, "tanh", "simt"),
         ((96, 130, 70, 10), 77, "tanh", "bf16x6"),
         ((96, 130, 70, 10), 77, "identity", "auto"),
         ((64, 300, 1), 200, "tanh", "tf32x3"),
         ((1100, 260, 20), 1030, "tanh", "auto"),      # BF16 x 2 terms where K >= 1024
         ((33, 7), 5, "tanh", "bf16x9")]


@pytest.mark.parametrize("widths,batch,hidden,algo", CASES,
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_train_step_stagewise(widths, batch, hidden, algo):
    torch = torch_gpu()
    net, Ws, bs, X, Y, Xd, Yd = _setup(widths, batch, hidden, algo, seed=51 + batch)
    lr = 0.05
    loss = net.train_step(Xd, Yd, lr)
    torch.cuda.synchronize()
    L = len(Ws)
    _check_forward(net, Ws, bs, X, hidden, algo)
    Hs = [_np(h) for h in net.H]
    Gs = [_np(g) for g in net.G]
    # loss gradient and loss
    R = Hs[-1].astype(np.float64) - Y.astype(np.float64)
    want = R / batch
    tol = (2 * U + U * U) * np.abs(R) / batch + TINY
    assert np.all(np.abs(Gs[-1] - want) <= tol)
    E64 = float(np.sum(R * R) / (2 * batch))
    N = R.size
    assert abs(float(loss.item()) - E64) <= (N + 4) * U * E64 + TINY
    # backward products and tanh'
    for l in range(L - 1, 0, -1):
        P64, D = _gemm64("T", "N", 1.0, Ws[l], Gs[l])
        eP = _gemm_bound(algo, Ws[l].shape[0], D)
        if hidden == "tanh":
            h = Hs[l - 1].astype(np.float64)
            d = 1 - h * h
            want = P64 * d
            tol = (eP * (1 + U) ** 2 + (2 * U + U * U) * np.abs(P64)) * np.abs(d) + TINY
        else:
            want, tol = P64, eP + TINY
        err = np.abs(Gs[l - 1] - want)
        assert np.all(err <= tol), (l, float(np.max(err / tol)))
    # weight update: one GEMM W' = W - lr G prev^T
    prevs = [X] + Hs[:-1]
    for l in range(L):
        W1 = _np(net.W[l])
        C64, D = _gemm64("N", "T", -lr, Gs[l], prevs[l], 1.0, Ws[l])
        tol = _gemm_bound(algo, batch, D) + TINY
        err = np.abs(W1 - C64)
        assert np.all(err <= tol), (l, float(np.max(err / tol)))
        # bias update
        b1 = _np(net.b[l]).astype(np.float64)
        G = Gs[l].astype(np.float64)
        want = bs[l].astype(np.float64) - lr * G.sum(axis=1)
        tol = lr * batch * U * np.abs(G).sum(axis=1) + U * np.abs(want) + TINY
        assert np.all(np.abs(b1 - want) <= tol), l


def test_step_is_deterministic_and_matches_fp64_step_closely():
    """Two runs from the same state are bit-identical (fixed-order reductions);
    the whole step tracks the FP64 oracle's step (normwise, loose check)."""
    torch = torch_gpu()
    widths, batch, lr = (200, 150, 40), 120, 0.1
    outs = []
    for _ in range(2):
        net, Ws, bs, X, Y, Xd, Yd = _setup(widths, batch, "tanh", "auto", seed=60)
        loss = net.train_step(Xd, Yd, lr)
        torch.cuda.synchronize()
        outs.append([_np(w) for w in net.W] + [_np(b) for b in net.b] + [_np(loss)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    E, Hs, Gs, newW, newb = omlp.step(Ws, bs, X, Y, lr)
    assert abs(float(outs[0][-1][0]) - E) <= 1e-5 * E
    for l in range(2):
        dW_gpu = outs[0][l].astype(np.float64) - Ws[l]
        dW_64 = newW[l] - Ws[l]
        assert np.linalg.norm(dW_gpu - dW_64) <= 1e-3 * np.linalg.norm(dW_64)


def test_training_reduces_loss_on_a_teacher_task():
    """Fit a fixed random teacher network: 40 steps cut the loss by half."""
    torch = torch_gpu()
    widths, batch = (64, 128, 16), 256
    rng = np.random.default_rng(70)
    Tw = [rng.normal(0, 1 / np.sqrt(widths[l]), (widths[l + 1], widths[l])) for l in range(2)]
    Tb = [rng.normal(0, 0.1, widths[l + 1]) for l in range(2)]
    net, Ws, bs, X, _, Xd, Yd = _setup(widths, batch, "tanh", "auto", seed=71)
    Y = omlp.forward(Tw, Tb, X)[-1].astype(np.float32)
    Yd.copy_(torch.from_numpy(Y))
    losses = [float(net.train_step(Xd, Yd, 0.5).item()) for _ in range(40)]
    assert losses[-1] < 0.5 * losses[0], losses[::8]


def test_argument_errors():
    torch = torch_gpu()
    import ctypes
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    lib = _lib.load()
    w = (ctypes.c_int64 * 3)(8, 0, 4)                      # a zero width
    d = _lib.MlpDesc(2, w, 4, 1)
    out = ctypes.c_size_t(0)
    assert lib.gb_mlp_workspace_size(-1, ctypes.byref(d), 1, ctypes.byref(out)) == _lib.GB_ERR_ARG
    w2 = (ctypes.c_int64 * 3)(8, 5, 4)
    d2 = _lib.MlpDesc(2, w2, 4, 7)                         # bad activation
    assert lib.gb_mlp_workspace_size(-1, ctypes.byref(d2), 1, ctypes.byref(out)) == _lib.GB_ERR_ARG
    net = gb.MLP((8, 5, 4), 4)
    X = gb.colmajor(8, 4)
    Y = gb.colmajor(4, 4)
    small = net.ws_bytes - 256
    rc = lib.gb_mlp_train_step(net.h.h, -1, ctypes.byref(net.desc),
                               (ctypes.c_void_p * 2)(*[t.data_ptr() for t in net.W]),
                               (ctypes.c_void_p * 2)(*[t.data_ptr() for t in net.b]),
                               X.data_ptr(), Y.data_ptr(), 0.1,
                               (ctypes.c_void_p * 2)(*[t.data_ptr() for t in net.H]),
                               (ctypes.c_void_p * 2)(*[t.data_ptr() for t in net.G]),
                               net.loss.data_ptr(), net.workspace.data_ptr(), small, None)
    assert rc == _lib.GB_ERR_WORKSPACE
    with pytest.raises(ValueError):
        net.train_step(gb.colmajor(8, 5), Y, 0.1)           # wrong batch
