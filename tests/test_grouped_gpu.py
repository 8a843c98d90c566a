"""Grouped SGEMM: 2000 uneven problems in one persistent launch, checked per
problem against the oracle; CUDA-graph replay gives the eager bits."""
import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu import torch_gpu

pytestmark = pytest.mark.gpu


def _check_problem(p, got_storage, cols=None, algo="simt"):
    from _gpu import STANDARD_BOUND_MIN_K, split_extra
    C64, D = oracle.sgemm(p.ta, p.tb, p.m, p.n, p.k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta,
                          p.C, p.ldc, cols=cols)
    sub = got_storage[:p.m, :] if cols is None else got_storage[:p.m, cols]
    rep = oracle.err_report(sub, C64, D, p.k, extra=split_extra(algo, p.k))
    assert rep["max_ratio"] <= 1.0, (p.ta, p.tb, p.m, p.n, p.k, rep)
    if p.k >= STANDARD_BOUND_MIN_K[algo]:
        assert oracle.err_report(sub, C64, D, p.k)["max_ratio"] <= 1.0


@pytest.fixture(scope="module")
def group2000():
    torch_gpu()
    return wl.grouped_problems(2000, seed=4)


@pytest.mark.parametrize("algo", ("simt", "auto", "bf16x6"))
def test_grouped_2000_against_oracle(group2000, algo):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    probs = group2000
    buf, tuples, views = gb.upload_problems(probs)
    plan = gb.GroupedPlan(tuples, algo=algo)
    plan.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(8)
    full = set(rng.choice(len(probs), size=60, replace=False).tolist())
    for i, p in enumerate(probs):
        got = views[i].cpu().numpy()
        if i in full:
            _check_problem(p, got, algo="simt")
        else:
            cols = np.unique(rng.integers(0, p.n, size=min(p.n, 3)))
            _check_problem(p, got, cols=cols, algo="simt")
    plan.close()


def test_grouped_graph_replay_is_bit_identical(group2000):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    probs = group2000[:400]
    buf, tuples, views = gb.upload_problems(probs)
    saved = buf.clone()
    plan = gb.GroupedPlan(tuples)
    plan.run()
    torch.cuda.synchronize()
    eager = buf.clone()
    buf.copy_(saved)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run(stream=s)
    torch.cuda.synchronize()
    buf.copy_(saved)                      # capture did not run the kernels; start clean
    for _ in range(2):
        buf.copy_(saved)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(buf, eager)
    plan.close()


def test_grouped_edge_cases():
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    rng = np.random.default_rng(9)
    probs = [
        wl.make_problem("N", "N", 0, 5, 5, 1.0, 0.0, rng=rng),       # M = 0: nothing
        wl.make_problem("T", "N", 7, 9, 11, 0.0, 1.0, rng=rng),      # alpha 0, beta 1: untouched
        wl.make_problem("N", "T", 7, 9, 11, 0.0, -2.0, rng=rng),     # alpha 0: beta*C
        wl.make_problem("T", "T", 13, 1, 0, 1.0, 0.5, rng=rng),      # K = 0: beta*C
        wl.make_problem("N", "N", 1, 1, 1, 1.5, 0.0, rng=rng),
        wl.make_problem("N", "N", 300, 200, 150, -1.0, 0.25, rng=rng),
    ]
    probs[1].A[:] = np.nan
    probs[2].A[:] = np.nan
    probs[2].B[:] = np.nan
    buf, tuples, views = gb.upload_problems(probs)
    before = [v.cpu().numpy().copy() for v in views]
    plan = gb.GroupedPlan(tuples)
    plan.run()
    torch.cuda.synchronize()
    after = [v.cpu().numpy() for v in views]
    assert np.array_equal(after[1], before[1])
    assert np.array_equal(after[2], np.float32(-2.0) * before[2])
    assert np.array_equal(after[3], np.float32(0.5) * before[3])
    for i in (4, 5):
        _check_problem(probs[i], after[i])
    plan.close()
    # a bad problem is reported with its index and BLAS argument position
    bad = list(tuples)
    t = list(bad[4])
    t[8] = 0                              # lda = 0 < 1
    bad[4] = tuple(t)
    with pytest.raises(_lib.GBError) as ei:
        gb.GroupedPlan(bad)
    assert ei.value.code == -8 and ei.value.bad_index == 4
    # an empty group is valid and runs nothing
    empty = gb.GroupedPlan([])
    assert empty.run() == 0
    empty.close()


# K values on both sides of every split's threshold (16 for TF32 x 2 terms,
# 1024 for BF16 x 2 terms, 9 for BF16 x 3 terms with 6 products, 10 with 9).
MIXED_K = (1, 3, 4, 9, 15, 16, 40, 300, 1023, 1024, 1500, 2100)


@pytest.mark.parametrize("algo", ("auto", "tf32x3", "bf16x3", "bf16x6", "bf16x9", "fp16x3"))
def test_grouped_per_problem_split_meets_fp32_bound(algo):
    """The plan picks a split per problem by K: each problem's result meets the
    plain FP32 bound, whichever split was preferred (a problem below the
    preferred split's threshold takes BF16 x 3 terms, K < 9 the CUDA cores)."""
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    rng = np.random.default_rng(31)
    probs = []
    for i, k in enumerate(MIXED_K * 2):
        m, n = int(rng.integers(60, 300)), int(rng.integers(60, 300))
        ta, tb = "NT"[i % 2], "NT"[(i // 2) % 2]
        probs.append(wl.make_problem(ta, tb, m, n, k, float(rng.uniform(-2, 2)),
                                     float(rng.uniform(-2, 2)), rng=rng,
                                     dist="logu" if i % 3 == 0 else "uniform"))
    buf, tuples, views = gb.upload_problems(probs)
    plan = gb.GroupedPlan(tuples, algo=algo)
    plan.run()
    torch.cuda.synchronize()
    assert gb.default_handle().device_error() == (0, 0)
    for i, p in enumerate(probs):
        _check_problem(p, views[i].cpu().numpy(), algo="simt")
    plan.close()


@pytest.mark.parametrize("algo", ("tf32x3", "bf16x3", "bf16x9"))
def test_grouped_split_integer_bit_exact(algo):
    """Integer data: every split and the mixed-mode plan are exact."""
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    rng = np.random.default_rng(32)
    probs = [wl.make_problem("NT"[i % 2], "TN"[i % 2], 100 + 13 * i, 90 + 7 * i, k, 1.0, 0.5,
                             rng=rng, dist="int") for i, k in enumerate((5, 20, 1100, 2048))]
    buf, tuples, views = gb.upload_problems(probs)
    plan = gb.GroupedPlan(tuples, algo=algo)
    plan.run()
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        C64, _ = oracle.sgemm(p.ta, p.tb, p.m, p.n, p.k, p.alpha, p.A, p.lda, p.B, p.ldb,
                              p.beta, p.C, p.ldc)
        got = views[i].cpu().numpy()[:p.m, :]
        assert np.array_equal(got, C64.astype(np.float32)), (algo, p.k)
    plan.close()
