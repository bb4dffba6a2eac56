"""Differentiable top-K search: torch.autograd.Function over knn_search and
knn_backward (argument marshalling only; both directions run in
libtpuknn.so).

The forward returns the K selected values (reported form: IP <q,x>, L2
||q - x||^2, COS the cosine) and their int32 indices. Selection is discrete:
the indices are not differentiable and stay fixed in the backward, which is
the gradient of sum_{i,k} g[i,k] * value(q_i, x_idx[i,k]) with respect to the
queries and the database rows (the scores of Sec. 2 differentiated
analytically; gather for dQ, scatter-add for dX).
"""
import torch

from .search import Database


class KnnTopK(torch.autograd.Function):
    """(val, idx) = search(q, db); gradients flow to q and to x, the FP32
    rows db was prepared from (x is only read by the backward)."""

    @staticmethod
    def forward(ctx, q, x, db, K, L, recall_target, rerank, bins, deterministic, exact):
        if exact:
            val, idx = db.search_exact(q.detach(), K)
        else:
            val, idx = db.search(q.detach(), K, L=L, recall_target=recall_target,
                                 rerank=rerank, bins=bins)
        ctx.db = db
        ctx.deterministic = bool(deterministic)
        ctx.save_for_backward(q, x, idx)
        ctx.mark_non_differentiable(idx)
        return val, idx

    @staticmethod
    def backward(ctx, g_val, g_idx):
        q, x, idx = ctx.saved_tensors
        want_q, want_x = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if g_val is None or not (want_q or want_x):
            return (None,) * 10
        dq, dx = ctx.db.backward(q.detach(), idx, g_val, want_dq=want_q, want_dx=want_x,
                                 deterministic=ctx.deterministic, x_f32=x.detach())
        return dq, dx, None, None, None, None, None, None, None, None


def knn_topk(q, x, db, K, L=None, recall_target=0.95, rerank=2, bins="mod",
             deterministic=False, exact=False):
    """Differentiable approximate (or exact) K-NN of the rows of q in db.

    q: M x D float32 CUDA tensor; x: the N x D float32 CUDA tensor db was
    built from (pass it with requires_grad=True to get dX); db: a Database.
    Returns (val M x K float32, idx M x K int32).
    """
    if not isinstance(db, Database):
        raise TypeError("db must be a Database")
    if tuple(x.shape) != (db.N, db.D) or x.dtype != torch.float32 or not x.is_cuda:
        raise ValueError("x must be the N x D float32 CUDA rows the database was built from")
    if q.dim() != 2 or q.shape[1] != db.D or q.dtype != torch.float32 or not q.is_cuda:
        raise ValueError("q must be an M x D float32 CUDA tensor")
    return KnnTopK.apply(q.contiguous(), x.contiguous(), db, int(K), L, recall_target, rerank,
                         bins, deterministic, exact)
