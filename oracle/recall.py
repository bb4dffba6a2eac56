"""Recall law of the bin-wise PartialReduce (Sec. 5.1) in FP64.

Test infrastructure only.

* ``paper_expected_recall(L, K)`` is Eq. 13, ``((L-1)/L)^(K-1)``: the chance
  that a given top-K item shares its bin with no other top-K item.
* ``exact_expected_recall(N, L, K)`` is the expectation of the recall the
  algorithm actually reaches with bins ``j mod L`` when the top-K index set
  is a uniformly random K-subset of the N rows (exchangeable rows). A bin
  keeps its best member, so the recall equals the number of bins hit by the
  top-K set divided by K; a bin of size n is missed with probability
  C(N-n, K) / C(N, K). Eq. 13 counts a bin holding two top-K items as losing
  both, so it is a lower bound of this value.
* ``min_bins(K, r)`` is Eq. 14: the smallest L with Eq. 13 >= r;
  ``approx_bins(K, r)`` is its first-order form (K-1)/(1-r) (App. A.4).
"""
import math


def paper_expected_recall(L, K):
    """Eq. 13: ((L-1)/L)^(K-1)."""
    if K <= 1:
        return 1.0
    return ((L - 1.0) / L) ** (K - 1)


def bin_sizes(N, L):
    """Sizes of the bins j mod L over rows 0..N-1 (the balanced contiguous
    bins have the same sizes, so the recall law below covers both maps)."""
    base, extra = divmod(N, L)
    return [base + (1 if b < extra else 0) for b in range(L)]


def _miss_prob(N, n, K):
    """C(N-n, K) / C(N, K) as a product, exact in FP64 to rounding."""
    if N - n < K:
        return 0.0
    p = 1.0
    for t in range(K):
        p *= (N - n - t) / (N - t)
    return p


def exact_expected_recall(N, L, K):
    """E[#bins hit by a uniform random K-subset] / K for bins j mod L."""
    if K > N:
        raise ValueError("K > N")
    sizes = bin_sizes(N, L)
    # bins of equal size contribute equally: group them
    counts = {}
    for n in sizes:
        counts[n] = counts.get(n, 0) + 1
    hit = sum(c * (1.0 - _miss_prob(N, n, K)) for n, c in counts.items() if n > 0)
    return hit / K


def min_bins(K, r):
    """Eq. 14: smallest integer L >= 1 with ((L-1)/L)^(K-1) >= r."""
    if not (0.0 < r < 1.0):
        raise ValueError("recall target must lie in (0, 1)")
    if K <= 1:
        return 1
    L = max(1, math.ceil(1.0 / (1.0 - r ** (1.0 / (K - 1)))))
    while L > 1 and paper_expected_recall(L - 1, K) >= r:
        L -= 1
    while paper_expected_recall(L, K) < r:
        L += 1
    return L


def approx_bins(K, r):
    """App. A.4: L ~ (K-1)/(1-r) for r close to 1."""
    return (K - 1) / (1.0 - r)
