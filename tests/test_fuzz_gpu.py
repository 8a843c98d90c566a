"""Seeded random sweep: 120 problems with random M, N, K (1 to 700, and a few
long-K ones), transposes, leading-dimension padding, alpha and beta (zero
included, with NaN in the C that beta = 0 must not read) and algorithms,
each checked against the oracle's bound for its algorithm and for the
padding rows' canary."""
import numpy as np
import pytest

import workloads as wl
from _gpu import ALGOS, assert_within_bound, auto_algo, check_padding, run, torch_gpu

pytestmark = pytest.mark.gpu


def _cases(n=120, seed=77):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        m, nn = (int(x) for x in rng.integers(1, 700, 2))
        k = int(rng.integers(1, 700)) if i % 10 else int(rng.integers(1500, 5000))
        ta, tb = rng.choice(["N", "T"]), rng.choice(["N", "T"])
        alpha = float(rng.choice([0.0, 1.0, -0.5, rng.uniform(-2, 2)], p=[0.05, 0.3, 0.15, 0.5]))
        beta = float(rng.choice([0.0, 1.0, rng.uniform(-2, 2)], p=[0.3, 0.1, 0.6]))
        algo = str(rng.choice(list(ALGOS) + ["auto"]))
        pad = int(rng.integers(0, 9))
        dist = str(rng.choice(["uniform", "logu"]))
        out.append((i, m, nn, k, ta, tb, alpha, beta, algo, pad, dist))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: f"c{c[0]}")
def test_random_problem(case):
    torch_gpu()
    i, m, n, k, ta, tb, alpha, beta, algo, pad, dist = case
    p = wl.make_problem(ta, tb, m, n, k, alpha, beta, seed=1000 + i, dist=dist, ld_pad=pad)
    if beta == 0.0:
        p.C[:m, :n] = np.nan                    # not read when beta = 0
    rc, got = run(p, algo)
    assert rc == 0
    check = algo
    if algo == "auto":
        check = auto_algo(k)
    assert_within_bound(p, got, algo=check)
    check_padding(p, got)
