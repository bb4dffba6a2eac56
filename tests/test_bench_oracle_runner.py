"""bench.py's CPU oracle baseline (and reference arm) on the CPU: the rows it
times against are stored exactly as the parity tests store them, and a run
advances through the query sample."""
import numpy as np
import pytest

import bench
from tests.test_gpu_lowp import stored


@pytest.mark.parametrize("dtype,metric", [("bf16", "l2"), ("e4m3", "cos"), ("f32", "ip"),
                                          ("bf16", "cos")])
def test_oracle_runner_stores_rows_like_the_parity_tests(dtype, metric):
    g = np.random.Generator(np.random.PCG64(5))
    X = g.standard_normal((600, 24)).astype(np.float32)
    Q = g.standard_normal((9, 24)).astype(np.float32)
    r = bench.OracleRunner(dict(X=X, Q=Q, metric=metric, dtype=dtype), L=64, K=5, rerank=3)
    if dtype == "f32":
        Xs = Xf = X.astype(np.float64)
    else:
        Xs, Xf = stored(X, metric, dtype)
    np.testing.assert_array_equal(r.Xs, Xs)
    np.testing.assert_array_equal(r.Xf, Xf)
    assert r.metric == ("ip" if metric == "cos" else metric)
    assert r.run(4) > 0 and r.cursor == 4
    assert r.run(7) > 0 and r.cursor == 2          # wraps around the 9 queries


def test_oracle_runner_without_rerank():
    g = np.random.Generator(np.random.PCG64(6))
    X = g.standard_normal((500, 16)).astype(np.float32)
    Q = g.standard_normal((5, 16)).astype(np.float32)
    r = bench.OracleRunner(dict(X=X, Q=Q, metric="ip", dtype="f32"), L=32, K=4, rerank=0)
    assert r.run(5) > 0 and r.cursor == 0
