"""Pins for the FP64 training-step oracle (oracle/mlp.py), fixed by calculus and
closed forms rather than by the oracle itself:

  * central finite differences of the loss, entry by entry, give dE/dW and dE/db;
  * a single linear layer has the closed-form least-squares gradient;
  * with identity hidden activations the network collapses to one affine map;
  * lr = 0 leaves the parameters unchanged, and a perfect fit has zero loss
    and zero gradients.

Planted mistakes (a dropped 1/B, tanh' taken from Z instead of H, a missing
transpose in the backward product, a dropped bias gradient) each fail a pin.
"""
import numpy as np
import pytest

from oracle import mlp

WIDTHS = (5, 7, 6, 3)
B = 4


def _net(seed, widths=WIDTHS, batch=B):
    rng = np.random.default_rng(seed)
    Ws = [rng.normal(0, 0.7, (widths[l + 1], widths[l])) for l in range(len(widths) - 1)]
    bs = [rng.normal(0, 0.3, widths[l + 1]) for l in range(len(widths) - 1)]
    X = rng.normal(0, 1, (widths[0], batch))
    Y = rng.normal(0, 1, (widths[-1], batch))
    return Ws, bs, X, Y


def _fd_check(Ws, bs, X, Y, hidden, h=1e-5):
    E, Hs, Gs, dWs, dbs = mlp.grads(Ws, bs, X, Y, hidden)
    rng = np.random.default_rng(1)
    worst = 0.0
    for l in range(len(Ws)):
        for _ in range(6):
            i, j = rng.integers(0, Ws[l].shape[0]), rng.integers(0, Ws[l].shape[1])
            Wp = [W.copy() for W in Ws]
            Wm = [W.copy() for W in Ws]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            fd = (mlp.loss(Wp, bs, X, Y, hidden) - mlp.loss(Wm, bs, X, Y, hidden)) / (2 * h)
            worst = max(worst, abs(fd - dWs[l][i, j]) / max(1e-3, abs(fd)))
        for i in range(Ws[l].shape[0]):
            bp = [b.copy() for b in bs]
            bm = [b.copy() for b in bs]
            bp[l][i] += h
            bm[l][i] -= h
            fd = (mlp.loss(Ws, bp, X, Y, hidden) - mlp.loss(Ws, bm, X, Y, hidden)) / (2 * h)
            worst = max(worst, abs(fd - dbs[l][i]) / max(1e-3, abs(fd)))
    return worst


@pytest.mark.parametrize("hidden", mlp.HIDDEN)
def test_gradients_match_central_differences(hidden):
    Ws, bs, X, Y = _net(0)
    assert _fd_check(Ws, bs, X, Y, hidden) < 1e-6


def test_single_linear_layer_closed_form():
    rng = np.random.default_rng(2)
    W = rng.normal(0, 1, (3, 5))
    b = rng.normal(0, 1, 3)
    X = rng.normal(0, 1, (5, 7))
    Y = rng.normal(0, 1, (3, 7))
    lr = 0.125
    R = W @ X + b[:, None] - Y
    E, Hs, Gs, newW, newb = mlp.step([W], [b], X, Y, lr)
    assert np.allclose(E, np.sum(R ** 2) / 14, rtol=1e-14, atol=0)
    assert np.allclose(newW[0], W - lr * R @ X.T / 7, rtol=1e-14, atol=1e-15)
    assert np.allclose(newb[0], b - lr * R.sum(axis=1) / 7, rtol=1e-14, atol=1e-15)


def test_identity_hidden_collapses_to_one_affine_map():
    Ws, bs, X, Y = _net(3)
    Hs = mlp.forward(Ws, bs, X, hidden="identity")
    M = Ws[2] @ Ws[1] @ Ws[0]
    c = Ws[2] @ (Ws[1] @ bs[0] + bs[1]) + bs[2]
    assert np.allclose(Hs[-1], M @ X + c[:, None], rtol=1e-12, atol=1e-12)


def test_tanh_layers_saturate_and_output_is_affine():
    Ws, bs, X, Y = _net(4)
    Hs = mlp.forward(Ws, bs, X, hidden="tanh")
    for H in Hs[:-1]:
        assert np.all(np.abs(H) < 1)
    assert np.allclose(Hs[-1], Ws[-1] @ Hs[-2] + bs[-1][:, None], rtol=1e-14, atol=1e-14)


def test_zero_learning_rate_and_perfect_fit():
    Ws, bs, X, _ = _net(5)
    Y = mlp.forward(Ws, bs, X)[-1]
    E, Hs, Gs, newW, newb = mlp.step(Ws, bs, X, Y, lr=0.0)
    assert E == 0.0
    for G in Gs:
        assert np.all(G == 0)
    for a, b in zip(newW + newb, Ws + bs):
        assert np.array_equal(a, b)


# ------------------------------------------------------ planted mistakes --

def _all_pins_pass():
    try:
        test_gradients_match_central_differences("tanh")
        test_gradients_match_central_differences("identity")
        test_single_linear_layer_closed_form()
        test_identity_hidden_collapses_to_one_affine_map()
        test_tanh_layers_saturate_and_output_is_affine()
        test_zero_learning_rate_and_perfect_fit()
    except AssertionError:
        return False
    return True


def _grads_no_inv_batch(Ws, bs, X, Y, hidden="tanh"):
    E, Hs, Gs, dWs, dbs = _orig_grads(Ws, bs, X, Y, hidden)
    B_ = np.asarray(X).shape[1]
    return E, Hs, [G * B_ for G in Gs], [d * B_ for d in dWs], [d * B_ for d in dbs]


def _grads_no_bias(Ws, bs, X, Y, hidden="tanh"):
    E, Hs, Gs, dWs, dbs = _orig_grads(Ws, bs, X, Y, hidden)
    return E, Hs, Gs, dWs, [np.zeros_like(d) for d in dbs]


_orig_grads = mlp.grads


@pytest.mark.parametrize("mistake", ["phi_from_z", "no_transpose", "no_inv_batch", "no_bias"])
def test_planted_mistakes_fail_a_pin(monkeypatch, mistake):
    assert _all_pins_pass()
    if mistake == "phi_from_z":
        # tanh' evaluated as 1 - Z^2 on the pre-activation (recovered as arctanh H)
        monkeypatch.setattr(mlp, "_phi_grad_from_output",
                            lambda kind, H: 1.0 - np.arctanh(H) ** 2 if kind == "tanh"
                            else np.ones_like(H))
    elif mistake == "no_transpose":
        def grads_wrong(Ws, bs, X, Y, hidden="tanh"):
            Ws = [np.asarray(W, dtype=np.float64) for W in Ws]
            E, Hs, Gs, dWs, dbs = _orig_grads(Ws, bs, X, Y, hidden)
            L = len(Ws)
            Gs = list(Gs)
            for l in range(L - 2, -1, -1):
                W = Ws[l + 1]
                # W instead of W^T (shapes permitting: pad/crop to fit)
                P = np.zeros((W.shape[1], W.shape[0]))
                r, c = min(P.shape[0], W.shape[0]), min(P.shape[1], W.shape[1])
                P[:r, :c] = W[:r, :c]
                Gs[l] = (P @ Gs[l + 1]) * mlp._phi_grad_from_output(hidden, Hs[l])
            prev = [np.asarray(X, dtype=np.float64)] + Hs[:-1]
            dWs = [Gs[l] @ prev[l].T for l in range(L)]
            dbs = [Gs[l].sum(axis=1) for l in range(L)]
            return E, Hs, Gs, dWs, dbs
        monkeypatch.setattr(mlp, "grads", grads_wrong)
    elif mistake == "no_inv_batch":
        monkeypatch.setattr(mlp, "grads", _grads_no_inv_batch)
    elif mistake == "no_bias":
        monkeypatch.setattr(mlp, "grads", _grads_no_bias)
    assert not _all_pins_pass()
