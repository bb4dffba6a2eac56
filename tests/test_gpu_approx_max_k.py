"""The approx_max_k / approx_min_k operator on a given score matrix against
the FP64 oracle: bit-exact values (the inputs are FP32 or BF16 numbers) and
indices, for both bin maps, with and without aggregation to top-K."""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_14286_gb300 import search as S
from tests.gpu_util import ensure_built

pytestmark = pytest.mark.gpu


def scores(M, N, seed, ties=True):
    g = np.random.Generator(np.random.PCG64(seed))
    X = g.standard_normal((M, N)).astype(np.float32)
    if ties:
        # repeated values and zeros of both signs exercise the tie rule
        X[:, ::7] = np.round(X[:, ::7])
        X[:, 3::11] = -0.0
    return X


@pytest.mark.parametrize("bins", ["mod", "contiguous"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_approx_max_k_matches_oracle(bins, dtype):
    ensure_built()
    M, N, K = 37, 5003, 10
    X = scores(M, N, 41)
    t = torch.from_numpy(X).cuda()
    if dtype == "bf16":
        t = t.to(torch.bfloat16)
    Xo = t.float().cpu().numpy().astype(np.float64)
    for L in (1, 7, 128, 1000, N):
        for is_min in (False, True):
            for agg in (False, True):
                k = min(K, L)
                v, i = S.approx_max_k(t, k, L=L, bins=bins, is_min=is_min, aggregate_to_topk=agg)
                ov, oi = oracle.approx_max_k(Xo, k, L, bins=bins, is_min=is_min,
                                             aggregate_to_topk=agg)
                v, i = v.cpu().numpy(), i.cpu().numpy()
                assert np.array_equal(i, oi), (L, is_min, agg)
                assert np.array_equal(v.astype(np.float64), ov), (L, is_min, agg)


def test_approx_max_k_many_rows_and_planned_bins():
    ensure_built()
    M, N, K = 70000, 64, 4                      # more rows than one grid dimension holds
    X = scores(M, N, 42)
    t = torch.from_numpy(X).cuda()
    v, i = S.approx_max_k(t, K, L=8)
    ov, oi = oracle.approx_max_k(X.astype(np.float64), K, 8)
    assert np.array_equal(i.cpu().numpy(), oi)
    # L from the recall law, and from a larger planning size (a shard of a
    # bigger input): the output width follows the planned L
    L1 = S.plan_bins(N, K, 0.9)
    v, i = S.approx_max_k(t[:50], K, recall_target=0.9, aggregate_to_topk=False)
    assert v.shape == (50, min(L1, N))
    L2 = min(S.plan_bins(10 * N, K, 0.99), N)
    v, i = S.approx_max_k(t[:50], K, recall_target=0.99, planning_size=10 * N,
                          aggregate_to_topk=False)
    assert v.shape == (50, L2)
    ov, oi = oracle.approx_max_k(X[:50].astype(np.float64), K, L2, aggregate_to_topk=False)
    assert np.array_equal(i.cpu().numpy(), oi)


@pytest.mark.parametrize("bins", ["mod", "contiguous"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("N", [4096, 5000, 70000])
def test_approx_max_k_16_byte_loads_match_oracle(bins, dtype, N):
    """L (j mod L bins) and N multiples of the columns one 16-byte load holds
    (4 FP32, 8 BF16): the vectorised kernels, bit-exact against the oracle
    including ties and zeros of both signs, rows, grid rows and column runs
    split over many CTAs (70000 columns span several CTAs of a row)."""
    ensure_built()
    M, K = 37, 10
    X = scores(M, N, 43)
    t = torch.from_numpy(X).cuda()
    if dtype == "bf16":
        t = t.to(torch.bfloat16)
    Xo = t.float().cpu().numpy().astype(np.float64)
    for L in (8, 64, 1000, N):
        for is_min in (False, True):
            for agg in (False, True):
                k = min(K, L)
                v, i = S.approx_max_k(t, k, L=L, bins=bins, is_min=is_min, aggregate_to_topk=agg)
                ov, oi = oracle.approx_max_k(Xo, k, L, bins=bins, is_min=is_min,
                                             aggregate_to_topk=agg)
                v, i = v.cpu().numpy(), i.cpu().numpy()
                assert np.array_equal(i, oi), (L, is_min, agg)
                assert np.array_equal(v.astype(np.float64), ov), (L, is_min, agg)
