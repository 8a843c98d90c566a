"""GPU checks of the autotuner and its record: every grouped tensor-core
configuration the tuner can choose (forced through the record) and both row
widths of the one-GEMM kernel give results within the bound against the
oracle; the tuners fill the record; a record for another device is refused;
a new handle loads the cache named by GB_SGEMM_TUNING in a fresh process."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import workloads as wl
from _gpu import STANDARD_BOUND_MIN_K, assert_within_bound, run, split_extra, torch_gpu

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _check(p, got, algo):
    C64, D = oracle.sgemm(p.ta, p.tb, p.m, p.n, p.k, p.alpha, p.A, p.lda, p.B, p.ldb, p.beta,
                          p.C, p.ldc)
    sub = got[:p.m, :]
    assert oracle.err_report(sub, C64, D, p.k, extra=split_extra(algo, p.k))["max_ratio"] <= 1.0
    if p.k >= STANDARD_BOUND_MIN_K[algo]:
        assert oracle.err_report(sub, C64, D, p.k)["max_ratio"] <= 1.0


@pytest.fixture(scope="module")
def group():
    torch_gpu()
    # 48 uneven problems over every size class, both transposes, alpha and beta
    return wl.grouped_problems(48, seed=21, lo=8, hi=700)


@pytest.mark.parametrize("algo", ("bf16x6", "tf32x3", "bf16x3", "bf16x9"))
@pytest.mark.parametrize("config", (0, 1, 2))
def test_every_grouped_configuration_within_bound(group, config, algo):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    h = gb.Handle()
    t = h.tuning()
    t.grouped_valid = 1
    for c in range(8):
        t.grouped_route[c] = 2 + config        # every class on the tensor cores, this config
    h.set_tuning(t)
    buf, tuples, views = gb.upload_problems(group)
    plan = gb.GroupedPlan(tuples, algo=algo, handle=h)
    plan.run()
    torch.cuda.synchronize()
    for i, p in enumerate(group):
        a = algo if p.k >= STANDARD_BOUND_MIN_K[algo] or algo == "bf16x6" else "bf16x6"
        _check(p, views[i].cpu().numpy(), a if p.k >= STANDARD_BOUND_MIN_K["bf16x6"] else "simt")
    plan.close()
    assert h.device_error() == (0, 0)


def test_grouped_tuner_fills_the_record_and_plans_stay_in_bound(group):
    torch = torch_gpu()
    import paper_1912_04379_gb300 as gb
    h = gb.Handle()
    assert h.tuning().grouped_valid == 0 or os.environ.get("GB_SGEMM_TUNING")
    h.tune_grouped()
    t = h.tuning()
    assert t.grouped_valid == 1
    assert all(0 <= v <= 4 for v in t.grouped_route)
    buf, tuples, views = gb.upload_problems(group)
    plan = gb.GroupedPlan(tuples, algo="auto", handle=h)
    plan.run()
    torch.cuda.synchronize()
    for i, p in enumerate(group):
        _check(p, views[i].cpu().numpy(), "simt")    # AUTO meets the plain bound
    plan.close()


@pytest.mark.parametrize("algo", ("bf16x3", "bf16x6", "tf32x3"))
def test_both_row_widths_and_the_tuner(algo):
    import paper_1912_04379_gb300 as gb
    h = gb.Handle()
    m, n, k = 700, 900, 1300
    p = wl.make_problem("T", "N", m, n, k, 1.5, -0.5, seed=22, ld_pad=3)
    outs = {}
    for rb in (64, 128):
        t = h.tuning()
        t.n_gemm = 1
        g = t.gemm[0]
        mode = {"tf32x3": 0, "bf16x3": 1, "bf16x6": 2}[algo]
        g.mode, g.log2_m, g.log2_n, g.log2_k, g.row_bytes = mode, 9, 9, 10, rb
        h.set_tuning(t)
        rc, got = run(p, algo, handle=h)
        assert rc == 0
        assert_within_bound(p, got, algo=algo)
        outs[rb] = got
    h.tune_sgemm(algo, "T", "N", m, n, k)
    t = h.tuning()
    assert t.n_gemm == 1 and t.gemm[0].row_bytes in (64, 128)
    rc, got = run(p, algo, handle=h)
    assert np.array_equal(got, outs[t.gemm[0].row_bytes])   # the recorded width is the one used


def test_record_for_another_device_is_refused():
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    h = gb.Handle()
    t = h.tuning()
    t.sm_count += 1
    rc = h.lib.gb_set_tuning(h.h, ctypes.byref(t))
    assert rc == _lib.GB_ERR_ARG
    t = h.tuning()
    t.grouped_route[0] = 9                    # not a routing value
    assert h.lib.gb_set_tuning(h.h, ctypes.byref(t)) == _lib.GB_ERR_ARG


def test_new_handle_loads_the_cache_named_by_the_environment(tmp_path):
    import paper_1912_04379_gb300 as gb
    from paper_1912_04379_gb300 import _lib
    h = gb.Handle()
    t = h.tuning()
    t.grouped_valid = 1
    for c in range(8):
        t.grouped_route[c] = (0, 1, 2, 3, 4, 2, 3, 4)[c]
    path = str(tmp_path / "cache.json")
    assert h.lib.gb_tuning_write(ctypes.byref(t), path.encode()) == 0
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_1912_04379_gb300 as gb\n"
            "t = gb.Handle().tuning()\n"
            "print(t.grouped_valid, list(t.grouped_route))\n" % ROOT)
    env = dict(os.environ, GB_SGEMM_TUNING=path)
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip().splitlines()[-1] == "1 [0, 1, 2, 3, 4, 2, 3, 4]"
