"""Softmax-over-top-K loss used to exercise the backward pass, in FP64.

Test infrastructure only.

For one query with selected scores s_1..s_K, temperature tau and a target
vector t: loss = sum_k t_k * p_k with p = softmax(s / tau). Its gradient
with respect to the scores is  dloss/ds_k = p_k (t_k - sum_m t_m p_m) / tau.
The total loss sums over queries.
"""
import numpy as np


def softmax_rows(s, tau):
    z = np.asarray(s, np.float64) / tau
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def loss(s, t, tau=0.1):
    p = softmax_rows(s, tau)
    return float((np.asarray(t, np.float64) * p).sum())


def loss_grad(s, t, tau=0.1):
    """d loss / d s, same shape as s."""
    p = softmax_rows(s, tau)
    t = np.asarray(t, np.float64)
    inner = (t * p).sum(axis=1, keepdims=True)
    return p * (t - inner) / tau
