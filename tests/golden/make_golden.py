"""Writes tests/golden/recall_law.txt from the oracle (oracle/recall.py only).

Each line: N K recall_target L=min_bins(K, r) (Eq. 14), Eq. 13 at that L, and
the exact expected recall of bins j mod L (the oracle's recall law).
Run:  python tests/golden/make_golden.py
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import recall as R  # noqa: E402

CASES = [  # (N, K, r): the search workloads' sizes
    (16384, 10, 0.95),
    (1_000_000, 10, 0.95),
    (10_000_000, 100, 0.95),
    (1_000_000, 32, 0.95),
    (4_000_000, 100, 0.95),
    (1_048_576, 10, 0.99),
]

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "recall_law.txt")
    with open(out, "w") as f:
        f.write("# N K r L paper_recall(Eq.13) exact_recall  -- written by make_golden.py\n")
        for N, K, r in CASES:
            L = R.min_bins(K, r)
            f.write("%d %d %.4f %d %.12f %.12f\n" % (N, K, r, L, R.paper_expected_recall(L, K),
                                                    R.exact_expected_recall(N, L, K)))
    print(open(out).read())
