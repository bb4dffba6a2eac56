"""knn_search_static: the search in the library's own scratch buffer.

The GPU tests call it through the C ABI twice in a row and compare each
result with knn_search (caller workspace) on the same inputs. Both run the
same kernels in the same order, so the indices must agree exactly and the
values to 1e-6 relative (they are expected to be identical). The file is
named to be collected last so that it also runs after every other test has
used the device; it passes alone in a fresh process as well.
"""

import pytest
import torch

from paper_2206_14286_gb300 import _lib
from paper_2206_14286_gb300 import build as B

CAP = _lib.STATIC_WORKSPACE_BYTES


def lib():
    B.build()
    return _lib.get()


def call_static(L_, args):
    return L_.knn_search_static(*args)


def test_header_capacity_matches_binding():
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "tpuknn.h")).read()
    m = re.search(r"#define KNN_STATIC_WORKSPACE_BYTES \((\d+)u << (\d+)\)", text)
    assert m and int(m.group(1)) << int(m.group(2)) == CAP


def test_rejections_happen_before_any_cuda_call():
    f = lib().knn_search_static
    # (db, scale, hnorm, f32, N, D, dtype, metric, q, M, K, L, bins, r, rerank, val, idx, stream)
    base = [None, None, None, None, 100, 8, 1, 1, None, 4, 3, 10, 0, 0.95, 2, None, None, None]

    def with_(**kw):
        a = list(base)
        pos = {"N": 4, "D": 5, "dt": 6, "me": 7, "M": 9, "K": 10, "L": 11, "bm": 12}
        for k, v in kw.items():
            a[pos[k]] = v
        return f(*a)

    assert with_(M=0) == _lib.KNN_OK                      # empty batch: no-op
    assert with_(me=9) == _lib.KNN_EINVAL
    assert with_(K=11, L=10) == _lib.KNN_EINVAL
    assert with_() == _lib.KNN_EINVAL                     # NULL pointers
    # a batch whose scratch exceeds the static buffer is refused up front
    big_m = 1 << 22
    need = lib().knn_search_workspace(10 ** 6, 128, 1, 1, big_m, 10, 256, 0, 0.95, 2)
    assert need > CAP
    assert with_(N=10 ** 6, D=128, M=big_m, K=10, L=256) == _lib.KNN_ENOMEM


CASES = [
    # (N, D, M, K, L, dtype, metric, bins)
    (300_000, 128, 1024, 10, 256, "bf16", "l2", "mod"),
    (300_000, 128, 1024, 10, 256, "bf16", "l2", "contiguous"),
    (50_000, 96, 200, 10, 128, "f32", "ip", "mod"),
    (70_001, 128, 513, 16, 384, "e4m3", "cos", "mod"),
]


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-%s-%s" % (c[5], c[6], c[7]))
def test_static_matches_workspace_search_twice(case):
    from paper_2206_14286_gb300 import search as S
    N, D, M, K, L, dtype, metric, bins = case
    L_ = lib()
    assert torch.cuda.is_available()
    need = L_.knn_search_workspace(N, D, _lib.DTYPE[dtype], _lib.METRIC[metric], M, K, L,
                                   _lib.BINS[bins], 0.95, 2)
    assert 0 < need <= CAP
    g = torch.Generator(device="cpu").manual_seed(1234 + N)
    X = torch.randn(N, D, generator=g).cuda()
    Q = torch.randn(M, D, generator=g).cuda()
    db = S.Database(X, metric=metric, dtype=dtype)
    ref_v, ref_i = db.search(Q, K, L=L, bins=bins)
    torch.cuda.synchronize()

    val = torch.empty((M, K), dtype=torch.float32, device="cuda")
    idx = torch.empty((M, K), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    args = list(db._args()) + [Q.data_ptr(), M, K, L, _lib.BINS[bins], 0.95, 2,
                                val.data_ptr(), idx.data_ptr(), stream]
    for rep in range(2):
        val.fill_(float("nan"))
        idx.fill_(-7)
        if rep == 1:
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            alloc0 = torch.cuda.memory_allocated()
        st = call_static(L_, args)
        assert st == _lib.KNN_OK, _lib.get().knn_status_string(st)
        torch.cuda.synchronize()
        if rep == 1:
            # the second call allocated nothing on the device
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
        assert torch.equal(idx, ref_i), "rep %d: indices differ" % rep
        scale = ref_v.abs().max().item() + 1e-30
        err = (val - ref_v).abs().max().item()
        assert err <= 1e-6 * scale, "rep %d: max |dv| %g" % (rep, err)
    S.sync_status()


@pytest.mark.gpu
def test_static_binding_method_matches():
    from paper_2206_14286_gb300 import search as S
    lib()
    g = torch.Generator(device="cpu").manual_seed(7)
    X = torch.randn(20_000, 64, generator=g).cuda()
    Q = torch.randn(100, 64, generator=g).cuda()
    db = S.Database(X, metric="ip", dtype="bf16")
    a = db.search(Q, 5, L=64)
    b = db.search_static(Q, 5, L=64)
    torch.cuda.synchronize()
    assert torch.equal(a[1], b[1])
    assert torch.equal(a[0], b[0])
