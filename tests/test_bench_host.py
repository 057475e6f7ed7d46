"""Host-side pieces of bench.py's CPU baseline: the oracle evaluated over
several host threads (contiguous ranges, one per thread) gives the same bits
as one call over the whole stream, whatever the split."""
import os
import sys

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("threads", [1, 2, 3, 7])
def test_threaded_oracle_evaluation_equals_one_call(threads):
    sys.path.insert(0, ROOT)
    import bench
    f = {"kind": "lorentzian", "a": -10.0, "b": 10.0, "p": [1.0, 0.0, 1.0]}
    k = oracle.design(f, 300)
    v = oracle.values(f, k, "project")
    rng = np.random.default_rng(3)
    x = rng.uniform(-11.0, 11.0, 100003).astype(np.float32).astype(np.float64)
    x[:301] = k
    x[301] = np.nan
    got = bench.oracle_eval_threads(k, v, x, threads)
    ref = oracle.evaluate(k, v, x)
    assert np.array_equal(got, ref, equal_nan=True)


def test_host_threads_is_positive():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.host_threads() >= 1
