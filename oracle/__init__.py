"""Plain FP64 CPU oracle for the TPU-KNN search path (arXiv 2206.14286).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product path never does, and this package shares no code with
``paper_2206_14286_gb300`` (the CUDA library and its binding).

Contents
  * ``knn_oracle.c`` (built to ``_build/liborc.so``): exact K-NN (Eq. 1-2),
    PartialReduce (Alg. 1) with bins ``j mod L`` or contiguous runs,
    ExactRescoring (Sec. 5), the approx_max_k operator on a given score matrix
    (App. A.1), re-rank, the gradient of selected scores, and the input
    preparation (bfloat16 / E4M3 rounding with per-row or one database-wide
    scale, cosine normalisation).
  * ``recall.py``: the expected-recall law (Eq. 12-13 and its exact form) and
    the bin count from a recall target (Eq. 14, App. A.4).
  * ``loss.py``: the softmax-over-top-K loss and its gradient in FP64.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
except the score error of BF16/FP8 inputs against the original FP32 data,
which is only reported ("parity unpinned" for that report).
"""
from .core import (  # noqa: F401
    IP, L2, COS, METRICS,
    build, lib_path,
    exact_topk, partial_reduce, topk_pairs, binwise_topk, rerank, grad, score,
    bin_max, approx_max_k,
    bf16_round, e4m3_rows, e4m3_round, e4m3_scaled, e4m3_tensor, e4m3_tensor_scale,
    normalize_rows, set_threads,
)
from . import recall, loss  # noqa: F401
