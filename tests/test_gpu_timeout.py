"""Failure handling of the device-side waits, made to happen without a fault.

Every wait of the tensor-core kernels' pipelines is bounded. The test lowers
the limit to one nanosecond (knn_set_wait_limit_ns), so the first wait of a
search that does not complete at once runs out: that CTA raises its abort
flag, every role of it stops issuing work, waits (with the fixed limit) for
the copies and MMAs it has already issued, frees its tensor memory and
returns. The host then sees KNN_ETIMEOUT from knn_sync_status exactly once;
with the limit restored, the next search on the same device and context is
bit-identical to one that never timed out. Nothing here traps, faults or
waits without a bound.
"""
import numpy as np
import pytest
import torch

from paper_2206_14286_gb300 import _lib
from paper_2206_14286_gb300 import search as S
from tests.gpu_util import db, dev, ensure_built

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,metric,D", [("bf16", "l2", 128), ("bf16", "ip", 768),
                                            ("e4m3", "cos", 96)])
def test_wait_timeout_is_reported_once_then_searches_are_clean(dtype, metric, D):
    ensure_built()
    lib = _lib.get()
    g = np.random.Generator(np.random.PCG64(2024 + D))
    X = g.standard_normal((60013, D)).astype(np.float32)
    Q = g.standard_normal((700, D)).astype(np.float32)
    d = db(X, metric, dtype)
    qd = dev(Q)
    ref = d.search(qd, 10, L=512)
    torch.cuda.synchronize()
    assert lib.knn_sync_status() == _lib.KNN_OK
    try:
        _lib.check(lib.knn_set_wait_limit_ns(1), "knn_set_wait_limit_ns")
        d.search(qd, 10, L=512)            # its results are undefined
        torch.cuda.synchronize()
        status = lib.knn_sync_status()
    finally:
        _lib.check(lib.knn_set_wait_limit_ns(0), "knn_set_wait_limit_ns")
    assert status == _lib.KNN_ETIMEOUT, _lib.get().knn_status_string(status)
    assert lib.knn_sync_status() == _lib.KNN_OK          # reported once, then cleared
    for _ in range(2):
        again = d.search(qd, 10, L=512)
        torch.cuda.synchronize()
        assert lib.knn_sync_status() == _lib.KNN_OK
        assert torch.equal(ref[1], again[1]) and torch.equal(ref[0], again[0])
    S.sync_status()
