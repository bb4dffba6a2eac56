"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Every check here compares the oracle with something other than itself: a
library routine (NumPy sort/argmax, torch dtype conversion), a closed form,
brute force on tiny inputs, an invariant, or a number printed in the paper.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import recall as R
from oracle import loss as LS

METRICS = ["ip", "l2", "cos"]


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def numpy_scores(Q, X, metric):
    """Larger-is-better scores written with NumPy broadcasting."""
    Q = np.asarray(Q, np.float64)
    X = np.asarray(X, np.float64)
    if metric == "ip":
        return Q @ X.T
    if metric == "l2":
        diff = Q[:, None, :] - X[None, :, :]
        return -np.einsum("mnd,mnd->mn", diff, diff)
    qn = np.linalg.norm(Q, axis=1)[:, None]
    xn = np.linalg.norm(X, axis=1)[None, :]
    return (Q @ X.T) / (qn * xn)


def numpy_topk(S, K):
    """Top-K per row by (score desc, index asc) with np.lexsort."""
    out = []
    for row in S:
        order = np.lexsort((np.arange(row.size), -row))
        out.append(order[:K])
    return np.array(out)


def reported(S, metric):
    return -S if metric == "l2" else S


# ----------------------------------------------------------------------------
# Exact K-NN (Eq. 1-2)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("shape", [(5, 40, 7, 4), (3, 17, 1, 17), (8, 64, 33, 1)])
def test_exact_matches_numpy_sort(metric, shape):
    M, N, D, K = shape
    g = rng(10 + M + N)
    Q, X = g.standard_normal((M, D)), g.standard_normal((N, D))
    val, idx = oracle.exact_topk(Q, X, K, metric)
    S = numpy_scores(Q, X, metric)
    ref = numpy_topk(S, K)
    np.testing.assert_array_equal(idx, ref)
    refv = reported(np.take_along_axis(S, ref, 1), metric)
    np.testing.assert_allclose(val, refv, rtol=1e-12, atol=1e-12)


def test_exact_ties_go_to_smaller_index():
    g = rng(3)
    X = g.standard_normal((10, 4))
    X[7] = X[2]        # duplicate rows give equal scores
    X[9] = X[2]
    Q = X[2:3] * 3.0   # query aligned with the duplicates: they are the top
    for metric in METRICS:
        _, idx = oracle.exact_topk(Q, X, 3, metric)
        assert list(idx[0]) == [2, 7, 9], metric


@pytest.mark.parametrize("metric", METRICS)
def test_exact_permutation_invariance(metric):
    g = rng(4)
    Q, X = g.standard_normal((6, 9)), g.standard_normal((80, 9))
    perm = g.permutation(80)
    _, idx = oracle.exact_topk(Q, X, 7, metric)
    _, idxp = oracle.exact_topk(Q, X[perm], 7, metric)
    np.testing.assert_array_equal(perm[idxp], idx)


def test_exact_k_larger_than_n_pads():
    g = rng(5)
    val, idx = oracle.exact_topk(g.standard_normal((2, 3)), g.standard_normal((4, 3)), 6, "ip")
    assert (idx[:, 4:] == -1).all() and np.isnan(val[:, 4:]).all()
    assert sorted(idx[0, :4]) == [0, 1, 2, 3]


# ----------------------------------------------------------------------------
# PartialReduce (Alg. 1) and ExactRescoring (Sec. 5)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("metric", METRICS)
def test_partial_reduce_brute_force_every_L(metric):
    g = rng(6)
    M, N, D = 4, 23, 5
    Q, X = g.standard_normal((M, D)), g.standard_normal((N, D))
    S = numpy_scores(Q, X, metric)
    for L in range(1, N + 4):
        V, A = oracle.partial_reduce(Q, X, L, metric)
        for b in range(L):
            rows = np.arange(b, N, L)
            if rows.size == 0:
                assert (A[:, b] == -1).all() and np.isneginf(V[:, b]).all()
                continue
            best = rows[np.argmax(S[:, rows], axis=1)]  # argmax: first max = smaller j
            np.testing.assert_array_equal(A[:, b], best)
            np.testing.assert_allclose(V[:, b], S[np.arange(M), best], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("metric", METRICS)
def test_partial_reduce_contiguous_brute_force_every_L(metric):
    """Contiguous bins (Alg. 1's ShiftRight) against NumPy's balanced split."""
    g = rng(23)
    M, N, D = 4, 29, 5
    Q, X = g.standard_normal((M, D)), g.standard_normal((N, D))
    S = numpy_scores(Q, X, metric)
    for L in range(1, N + 1):
        V, A = oracle.partial_reduce(Q, X, L, metric, bins="contiguous")
        for b, rows in enumerate(np.array_split(np.arange(N), L)):
            best = rows[np.argmax(S[:, rows], axis=1)]
            np.testing.assert_array_equal(A[:, b], best)
            np.testing.assert_allclose(V[:, b], S[np.arange(M), best], rtol=1e-12, atol=1e-12)


def test_contiguous_power_of_two_is_shift_right():
    """When L divides N into runs of 2^W rows, the bin is j >> W (Alg. 1)."""
    g = rng(24)
    Q, X = g.standard_normal((3, 4)), g.standard_normal((64, 4))
    _, A = oracle.partial_reduce(Q, X, 8, "ip", bins="contiguous")
    assert np.all(A >> 3 == np.arange(8)[None, :])


@pytest.mark.parametrize("metric", METRICS)
def test_contiguous_L_equal_N_is_exact_and_recall_law(metric):
    g = rng(25)
    Q, X = g.standard_normal((9, 12)), g.standard_normal((150, 12))
    v1, i1 = oracle.binwise_topk(Q, X, 10, 150, metric, bins="contiguous")
    v2, i2 = oracle.exact_topk(Q, X, 10, metric)
    np.testing.assert_array_equal(i1, i2)


def test_empirical_recall_contiguous_bins():
    g = rng(26)
    N, D, M, K, L = 4096, 16, 400, 10, 60
    X, Q = g.standard_normal((N, D)), g.standard_normal((M, D))
    _, ie = oracle.exact_topk(Q, X, K, "ip")
    _, ib = oracle.binwise_topk(Q, X, K, L, "ip", bins="contiguous")
    rec = np.array([len(set(ie[i]) & set(ib[i])) / K for i in range(M)])
    sem = rec.std() / math.sqrt(M)
    assert abs(rec.mean() - R.exact_expected_recall(N, L, K)) < 5 * sem


def test_partial_reduce_tie_keeps_smaller_index():
    X = np.zeros((12, 3))
    X[:, 0] = 1.0                    # every row scores the same
    V, A = oracle.partial_reduce(np.ones((1, 3)), X, 5, "ip")
    np.testing.assert_array_equal(A[0], [0, 1, 2, 3, 4])


@pytest.mark.parametrize("metric", METRICS)
def test_binwise_with_L_equal_N_is_exact(metric):
    """With L = N every bin holds one row, so the method is exact (Alg. 1)."""
    g = rng(7)
    Q, X = g.standard_normal((9, 12)), g.standard_normal((150, 12))
    v1, i1 = oracle.binwise_topk(Q, X, 10, 150, metric)
    v2, i2 = oracle.exact_topk(Q, X, 10, metric)
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_allclose(v1, v2, rtol=1e-12)


@pytest.mark.parametrize("metric", METRICS)
def test_binwise_L1_K1_is_global_argmax(metric):
    g = rng(8)
    Q, X = g.standard_normal((7, 6)), g.standard_normal((90, 6))
    _, idx = oracle.binwise_topk(Q, X, 1, 1, metric)
    np.testing.assert_array_equal(idx[:, 0], np.argmax(numpy_scores(Q, X, metric), axis=1))


@pytest.mark.parametrize("metric", METRICS)
def test_binwise_results_are_bin_maxima(metric):
    g = rng(9)
    N, L = 500, 37
    Q, X = g.standard_normal((5, 8)), g.standard_normal((N, 8))
    S = numpy_scores(Q, X, metric)
    _, idx = oracle.binwise_topk(Q, X, 12, L, metric)
    for i in range(5):
        assert len(set(idx[i] % L)) == 12          # one winner per bin
        for j in idx[i]:
            rows = np.arange(j % L, N, L)
            assert S[i, j] == S[i, rows].max()
        # and the K winners are the best K among all L bin maxima
        maxima = np.array([S[i, np.arange(b, N, L)].max() for b in range(L)])
        assert np.isclose(np.sort(maxima)[::-1][:12], np.sort(S[i, idx[i]])[::-1]).all()


def test_topk_pairs_matches_numpy():
    g = rng(11)
    V = g.standard_normal((6, 40))
    A = g.permutation(1000)[:240].reshape(6, 40)
    A[0, 3] = -1                                   # an empty bin is skipped
    V[1, 5] = V[1, 6]                              # tie -> smaller index first
    val, idx = oracle.topk_pairs(V, A, 9)
    for i in range(6):
        ok = A[i] >= 0
        order = np.lexsort((A[i][ok], -V[i][ok]))[:9]
        np.testing.assert_array_equal(idx[i], A[i][ok][order])
        np.testing.assert_array_equal(val[i], V[i][ok][order])


@pytest.mark.parametrize("metric", METRICS)
def test_rerank_all_candidates_is_exact(metric):
    g = rng(12)
    Q, X = g.standard_normal((4, 10)), g.standard_normal((60, 10))
    cand = np.tile(g.permutation(60), (4, 1))
    v1, i1 = oracle.rerank(Q, X, cand, 5, metric)
    v2, i2 = oracle.exact_topk(Q, X, 5, metric)
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_allclose(v1, v2, rtol=1e-12)


# ----------------------------------------------------------------------------
# Metric identities: half-norm L2 (App. A.2, Eq. 15-19); cosine = MIPS on
# normalised rows (Sec. 2)
# ----------------------------------------------------------------------------
def test_half_norm_l2_ranking_identity():
    g = rng(13)
    Q, X = g.standard_normal((10, 16)), g.standard_normal((300, 16))
    _, idx = oracle.exact_topk(Q, X, 15, "l2")
    relaxed = 0.5 * (X * X).sum(1)[None, :] - Q @ X.T      # Eq. 19, argmin
    np.testing.assert_array_equal(idx, numpy_topk(-relaxed, 15))


def test_cosine_is_mips_on_normalised_rows():
    g = rng(14)
    Q, X = g.standard_normal((10, 16)), g.standard_normal((300, 16)) * 3.0
    vc, ic = oracle.exact_topk(Q, X, 15, "cos")
    Qn = Q / np.linalg.norm(Q, axis=1, keepdims=True)
    Xn = X / np.linalg.norm(X, axis=1, keepdims=True)
    vi, ii = oracle.exact_topk(Qn, Xn, 15, "ip")
    np.testing.assert_array_equal(ic, ii)
    np.testing.assert_allclose(vc, vi, rtol=1e-12)


# ----------------------------------------------------------------------------
# Recall law (Sec. 5.1, Eq. 12-14, App. A.4)
# ----------------------------------------------------------------------------
def test_exact_recall_closed_forms():
    assert R.exact_expected_recall(1000, 1000, 10) == pytest.approx(1.0, abs=1e-12)  # L = N
    assert R.exact_expected_recall(1000, 7, 1) == pytest.approx(1.0, abs=1e-12)      # K = 1
    # one bin: only one of the K items can be kept
    assert R.exact_expected_recall(500, 1, 8) == pytest.approx(1.0 / 8, abs=1e-12)
    # equal bins, large N: (L/K) (1 - (1 - 1/L)^K)
    L, K = 176, 10
    approx = (L / K) * (1.0 - (1.0 - 1.0 / L) ** K)
    assert R.exact_expected_recall(L * 20000, L, K) == pytest.approx(approx, rel=1e-5)
    # the paper's value is a lower bound
    for L, K in [(176, 10), (1931, 100), (605, 32), (1024, 10)]:
        assert R.paper_expected_recall(L, K) <= R.exact_expected_recall(10 ** 6, L, K)


def test_exact_recall_matches_monte_carlo():
    N, L, K, T = 300, 23, 9, 20000
    g = rng(15)
    hits = np.empty(T)
    for t in range(T):
        s = g.choice(N, size=K, replace=False)
        hits[t] = len(set((s % L).tolist())) / K
    sem = hits.std() / math.sqrt(T)
    assert abs(hits.mean() - R.exact_expected_recall(N, L, K)) < 5 * sem


def test_paper_recall_is_the_no_collision_probability():
    """Eq. 13 equals P(a given ball shares its bin with no other ball)."""
    L, K = 13, 6
    # brute force over the other K-1 balls' bins
    cnt = 0
    total = L ** (K - 1)
    for code in range(total):
        bins = []
        c = code
        for _ in range(K - 1):
            bins.append(c % L)
            c //= L
        cnt += 0 not in bins          # ball 0 sits in bin 0 by symmetry
    assert cnt / total == pytest.approx(R.paper_expected_recall(L, K), rel=1e-12)


def test_empirical_recall_on_random_data():
    """Bin-wise vs exact on i.i.d. rows: recall = the exact law within sampling error."""
    g = rng(16)
    N, D, M, K, L = 4096, 16, 400, 10, 60
    X, Q = g.standard_normal((N, D)), g.standard_normal((M, D))
    _, ie = oracle.exact_topk(Q, X, K, "ip")
    _, ib = oracle.binwise_topk(Q, X, K, L, "ip")
    rec = np.array([len(set(ie[i]) & set(ib[i])) / K for i in range(M)])
    sem = rec.std() / math.sqrt(M)
    expect = R.exact_expected_recall(N, L, K)
    assert abs(rec.mean() - expect) < 5 * sem
    assert rec.mean() > R.paper_expected_recall(L, K)


@pytest.mark.parametrize("K,r", [(10, 0.95), (100, 0.95), (32, 0.95), (10, 0.9), (2, 0.5), (50, 0.99)])
def test_min_bins_inverts_eq13(K, r):
    L = R.min_bins(K, r)
    assert R.paper_expected_recall(L, K) >= r
    assert L == 1 or R.paper_expected_recall(L - 1, K) < r
    assert L == math.ceil(1.0 / (1.0 - r ** (1.0 / (K - 1))) - 1e-9)


def test_min_bins_first_order_form():
    """App. A.4: L ~ (K-1)/(1-r); the relative gap shrinks as r -> 1."""
    gaps = []
    for r in [0.9, 0.95, 0.99, 0.999]:
        L = R.min_bins(10, r)
        gaps.append(abs(L - R.approx_bins(10, r)) / R.approx_bins(10, r))
    assert all(a >= b for a, b in zip(gaps, gaps[1:]))
    assert gaps[-1] < 1e-3
    assert R.min_bins(1, 0.99) == 1


# ----------------------------------------------------------------------------
# Gradient of selected scores, and the softmax loss
# ----------------------------------------------------------------------------
def _selected_value_sum(Q, X, idx, g, metric):
    S = reported(numpy_scores(Q, X, metric), metric)
    return float((np.take_along_axis(S, idx, 1) * g).sum())


@pytest.mark.parametrize("metric", METRICS)
def test_grad_central_differences(metric):
    gen = rng(17)
    M, N, D, K = 3, 12, 5, 4
    Q, X = gen.standard_normal((M, D)), gen.standard_normal((N, D))
    idx = np.stack([gen.permutation(N)[:K] for _ in range(M)])
    idx[1, 2] = idx[0, 0]                 # a row selected by two queries
    w = gen.standard_normal((M, K))
    dQ, dX = oracle.grad(Q, X, idx, w, metric)
    h = 1e-6
    for (A, dA) in [(Q, dQ), (X, dX)]:
        num = np.zeros_like(A)
        for t in range(A.size):
            a0 = A.flat[t]
            A.flat[t] = a0 + h
            fp = _selected_value_sum(Q, X, idx, w, metric)
            A.flat[t] = a0 - h
            fm = _selected_value_sum(Q, X, idx, w, metric)
            A.flat[t] = a0
            num.flat[t] = (fp - fm) / (2 * h)
        np.testing.assert_allclose(dA, num, rtol=1e-6, atol=1e-7)


def test_softmax_loss_grad_central_differences():
    gen = rng(18)
    s, t = gen.standard_normal((4, 6)), gen.standard_normal((4, 6))
    gr = LS.loss_grad(s, t, 0.1)
    h = 1e-7
    for k in range(s.size):
        sp, sm = s.copy(), s.copy()
        sp.flat[k] += h
        sm.flat[k] -= h
        num = (LS.loss(sp, t, 0.1) - LS.loss(sm, t, 0.1)) / (2 * h)
        assert gr.flat[k] == pytest.approx(num, rel=1e-5, abs=1e-6)


# ----------------------------------------------------------------------------
# Input preparation: bfloat16 and E4M3 rounding against torch's dtype
# conversions (library routines), cosine normalisation
# ----------------------------------------------------------------------------
def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    g = rng(19)
    x = (g.standard_normal(20000) * np.exp(g.uniform(-20, 20, 20000))).astype(np.float32)
    # exact ties in both parities, and values next to the overflow boundary
    base = np.array([1.0, 1.0078125, 3.0e38, -3.3e38, 1e-40], np.float32).view(np.uint32)
    extra = np.concatenate([(base & 0xFFFF0000) | 0x8000, (base & 0xFFFF0000) | 0x7FFF,
                            (base & 0xFFFF0000) | 0x8001]).view(np.float32)
    x = np.concatenate([x, extra, np.float32([0.0, -0.0, 65504.0])])
    ours = oracle.bf16_round(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ours, ref)


def test_e4m3_round_matches_torch_in_range():
    torch = pytest.importorskip("torch")
    g = rng(20)
    v = np.concatenate([g.uniform(-448, 448, 5000), g.standard_normal(5000) * 0.01,
                        np.arange(-448, 449, 0.0625), [2.0 ** -10, 3 * 2.0 ** -10, 2.0 ** -6]])
    v = v.astype(np.float32)
    ours = np.array([oracle.e4m3_round(t) for t in v])
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(ours, ref)


def test_e4m3_known_codes_and_saturation():
    assert oracle.e4m3_round(448.0) == 448.0
    assert oracle.e4m3_round(463.9) == 448.0       # would round to 448 anyway
    assert oracle.e4m3_round(1e9) == 448.0         # saturates, never inf
    assert oracle.e4m3_round(-500.0) == -448.0
    assert oracle.e4m3_round(2.0 ** -9) == 2.0 ** -9   # smallest subnormal
    assert oracle.e4m3_round(2.0 ** -11) == 0.0
    assert oracle.e4m3_round(1.0625) == 1.0        # tie to even (1.000)
    assert oracle.e4m3_round(1.1875) == 1.25       # tie to even (1.010)


def test_e4m3_rows_scale_and_range():
    g = rng(21)
    x = g.standard_normal((50, 24)).astype(np.float32)
    x[3] = 0.0
    deq, sc = oracle.e4m3_rows(x)
    assert sc[3] == 1.0 and (deq[3] == 0.0).all()
    mx = np.abs(x).max(axis=1)
    ok = mx > 0
    np.testing.assert_array_equal(sc[ok], (mx[ok] / np.float32(448.0)).astype(np.float32))
    # the largest element of each row lands on the top code, 448 * s
    am = np.abs(x).argmax(axis=1)
    top = np.abs(deq[np.arange(50), am])[ok]
    np.testing.assert_allclose(top, 448.0 * sc[ok].astype(np.float64), rtol=0)
    # relative error of every element is at most half a step (2^-4) or subnormal step
    err = np.abs(deq - x) / (sc[:, None].astype(np.float64))
    assert (err <= np.maximum(np.abs(x) / sc[:, None] * 2.0 ** -4, 2.0 ** -10) + 1e-12).all()


def test_normalize_rows_unit_norm():
    g = rng(22)
    x = (g.standard_normal((40, 96)) * 5).astype(np.float32)
    x[0] = 0
    y = oracle.normalize_rows(x)
    n = np.linalg.norm(y.astype(np.float64), axis=1)
    assert n[0] == 0.0
    np.testing.assert_allclose(n[1:], 1.0, atol=1e-6)
    x64 = x[1:].astype(np.float64)
    ref = x64 / np.linalg.norm(x64, axis=1, keepdims=True)
    np.testing.assert_allclose(y[1:], ref, rtol=1e-6, atol=1e-7)


# ----------------------------------------------------------------------------
# Stored oracle outputs written by tests/golden/make_golden.py
# ----------------------------------------------------------------------------
def test_recall_law_golden_file():
    path = os.path.join(os.path.dirname(__file__), "golden", "recall_law.txt")
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        N, K, r, L, paper, exact = line.split()
        N, K, L = int(N), int(K), int(L)
        assert R.min_bins(K, float(r)) == L
        assert R.paper_expected_recall(L, K) == pytest.approx(float(paper), rel=1e-9)
        assert R.exact_expected_recall(N, L, K) == pytest.approx(float(exact), rel=1e-9)


# ----------------------------------------------------------------------------
# approx_max_k on a given score matrix (App. A.1)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("bins", ["mod", "contiguous"])
def test_bin_max_brute_force_every_L(bins):
    g = np.random.Generator(np.random.PCG64(31))
    M, N = 3, 11
    S = g.integers(-4, 5, size=(M, N)).astype(np.float64)   # many ties
    for L in range(1, N + 1):
        V, A = oracle.bin_max(S, L, bins)
        if bins == "mod":
            members = [np.arange(l, N, L) for l in range(L)]
        else:
            q, r = N // L, N % L
            members = [np.arange(l * q + min(l, r), (l + 1) * q + min(l + 1, r)) for l in range(L)]
        for i in range(M):
            for l in range(L):
                cols = members[l]
                j = cols[np.argmax(S[i, cols])]      # numpy keeps the first maximum
                assert A[i, l] == j and V[i, l] == S[i, j]


@pytest.mark.parametrize("bins", ["mod", "contiguous"])
def test_bin_max_equals_partial_reduce_on_ip_scores(bins):
    """Integer rows keep every FP64 score exact, so the two definitions meet."""
    g = np.random.Generator(np.random.PCG64(32))
    Q = g.integers(-3, 4, size=(5, 6)).astype(np.float64)
    X = g.integers(-3, 4, size=(40, 6)).astype(np.float64)
    for L in (1, 3, 7, 40):
        V1, A1 = oracle.bin_max(Q @ X.T, L, bins)
        V2, A2 = oracle.partial_reduce(Q, X, L, "ip", bins=bins)
        assert np.array_equal(A1, A2) and np.array_equal(V1, V2)


def test_approx_max_k_with_L_equal_N_is_exact_top_k():
    g = np.random.Generator(np.random.PCG64(33))
    S = g.standard_normal((4, 30))
    S[0, 5] = S[0, 9] = S[0].max() + 1.0          # a tie at the top: smaller index first
    for is_min in (False, True):
        v, a = oracle.approx_max_k(S, 6, 30, is_min=is_min)
        for i in range(4):
            order = np.lexsort((np.arange(30), S[i] if is_min else -S[i]))[:6]
            assert np.array_equal(a[i], order)
            assert np.array_equal(v[i], S[i, order])


def test_approx_max_k_bins_only_and_min_orientation():
    g = np.random.Generator(np.random.PCG64(34))
    S = g.standard_normal((3, 50))
    v, a = oracle.approx_max_k(S, 5, 8, aggregate_to_topk=False)
    assert v.shape == (3, 8) and np.all(a % 8 == np.arange(8))
    vmin, amin = oracle.approx_max_k(S, 5, 8, is_min=True, aggregate_to_topk=False)
    for i in range(3):
        for l in range(8):
            cols = np.arange(l, 50, 8)
            assert amin[i, l] == cols[np.argmin(S[i, cols])]
            assert vmin[i, l] == S[i, cols].min()


def test_e4m3_tensor_equals_rows_when_every_row_has_the_same_maximum():
    """With one maximum |x| shared by every row, the database-wide scale is
    each row's own scale: e4m3_tensor reduces to the pinned e4m3_rows."""
    g = rng(22)
    x = g.uniform(-1.0, 1.0, (40, 33)).astype(np.float32)
    x[:, 5] = np.where(g.random(40) < 0.5, 1.5, -1.5).astype(np.float32)
    deq_t, s = oracle.e4m3_tensor(x)
    deq_r, sc = oracle.e4m3_rows(x)
    assert (sc == s).all()
    np.testing.assert_array_equal(deq_t, deq_r)


def test_e4m3_tensor_matches_torch_cast():
    """Codes are torch's float8_e4m3fn cast of x / s (binary32 division)."""
    torch = pytest.importorskip("torch")
    g = rng(23)
    x = (g.standard_normal((64, 96)) * np.exp(g.uniform(-6, 2, (64, 1)))).astype(np.float32)
    x[7] = 0.0
    deq, s = oracle.e4m3_tensor(x)
    assert s == np.float32(np.abs(x).max()) / np.float32(448.0)
    q = torch.from_numpy(x) / torch.tensor(float(s), dtype=torch.float32)
    ref = q.to(torch.float8_e4m3fn).to(torch.float64).numpy() * np.float64(s)
    np.testing.assert_array_equal(deq, ref)
    # the largest |x| maps to the largest code, a zero row stays zero
    i = np.unravel_index(np.abs(x).argmax(), x.shape)
    assert abs(deq[i]) == 448.0 * np.float64(s)
    assert (deq[7] == 0.0).all()
    # a row much smaller than the largest keeps its relative precision
    # (E4M3 is floating point): its codes are still normal numbers
    rmax = np.abs(x).max(axis=1)
    small = np.where(rmax > 0, rmax, np.inf).argmin()
    assert rmax[small] < 1e-3 * rmax.max()
    nz = x[small] != 0
    rel = np.abs(deq[small][nz] - x[small][nz]) / np.abs(x[small][nz])
    assert rel[np.abs(x[small][nz]) / s >= 2.0 ** -6].max() <= 2.0 ** -4


def test_e4m3_tensor_scale_of_zero_database():
    assert oracle.e4m3_tensor_scale(np.zeros((3, 4), np.float32)) == 1.0
