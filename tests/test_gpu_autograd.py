"""The differentiable search (torch.autograd.Function over knn_search and
knn_backward) against the FP64 oracle and finite differences.

The loss is the softmax-over-top-K loss: sum_i sum_k t_ik softmax(v_i / 0.1)_k
with seeded targets t. On the GPU side torch differentiates the softmax and
the custom backward kernel takes d loss / d v; the oracle makes its own
selection, its own values and its own d loss / d v (oracle.loss) and its own
gradient (oracle.grad), all in FP64.

Gradients are compared only where the selection is the oracle's: queries whose
top-K margins exceed the selection tolerance (FP32 path) or whose returned
indices agree with the oracle's (low precision path), and database rows
touched only by such queries; every untouched row must be exactly zero.
Tolerance: 1e-4 of the largest gradient entry (FP32 accumulation over at most
K or M terms, the softmax evaluated in FP32).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import loss as OL
from paper_2206_14286_gb300 import synth
from paper_2206_14286_gb300.autograd import knn_topk
from tests import parity as PT
from tests.gpu_util import db, dev, host

pytestmark = pytest.mark.gpu
TAU = 0.1


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def gpu_loss(val, T):
    p = torch.softmax(val / TAU, dim=1)
    return (T * p).sum()


def oracle_exact(Q, X, K, metric):
    """Oracle selection (exact top-K, FP64) with the decided mask (FP32 tolerance)."""
    ov, oi = oracle.exact_topk(Q, X, K + 1, metric)
    S = PT.score_matrix(Q, X, metric)
    tol = PT.REL_F32 * PT.query_scale(Q, X, metric)
    srt = -np.sort(-S, axis=1)[:, :K + 1]
    gaps = srt[:, :-1] - srt[:, 1:]
    decided = (gaps > 2 * tol[:, None]).all(axis=1)
    return ov[:, :K], oi[:, :K], decided


def compare_grads(gdq, gdx, Q, X, oi, ov, T, metric, ok_q):
    """Oracle gradient for the selection oi (rows of ok_q only) vs the GPU's."""
    g = OL.loss_grad(ov, T, TAU)
    odq, odx = oracle.grad(Q, X, oi, g, metric)
    sq = np.abs(odq).max() + 1e-30
    np.testing.assert_allclose(gdq[ok_q], odq[ok_q], rtol=0, atol=1e-4 * sq)
    touched = np.zeros(X.shape[0], bool)
    touched[oi.reshape(-1)] = True
    bad = np.zeros(X.shape[0], bool)
    bad[oi[~ok_q].reshape(-1)] = True
    rows = touched & ~bad
    sx = np.abs(odx).max() + 1e-30
    np.testing.assert_allclose(gdx[rows], odx[rows], rtol=0, atol=1e-4 * sx)
    # rows no oracle query selected: zero unless an undecided query took them
    free = ~touched
    assert np.count_nonzero(gdx[free].any(axis=1)) <= int((~ok_q).sum()) * oi.shape[1]
    return rows.sum()


@pytest.mark.parametrize("metric", ["ip", "l2", "cos"])
def test_autograd_exact_f32_matches_oracle(metric):
    N, M, D, K = 3000, 48, 40, 8
    X = synth.iid_normal(N, D, 21, std=1.0 / np.sqrt(D))
    Q = synth.iid_normal(M, D, 22, std=1.0 / np.sqrt(D))
    T = synth.targets(M, K, seed=23)
    d = db(X, metric, "f32")
    xt = dev(X).requires_grad_(True)
    qt = dev(Q).requires_grad_(True)
    val, idx = knn_topk(qt, xt, d, K, exact=True)
    gpu_loss(val, dev(T)).backward()
    ov, oi, dec = oracle_exact(Q, X, K, metric)
    assert dec.mean() > 0.9
    gi = host(idx)
    assert np.array_equal(gi[dec], oi[dec])
    n = compare_grads(host(qt.grad), host(xt.grad), Q, X, oi, ov, T, metric, dec)
    assert n > 0


@pytest.mark.parametrize("metric", ["ip", "l2"])
def test_autograd_bf16_approx_matches_oracle(metric):
    """BF16 storage, bin-wise selection with FP32 re-rank; backward on FP32 rows."""
    N, M, D, K, L = 20000, 64, 64, 10, 128
    X = synth.mixture(N, D, 64, 31)
    Q = synth.mixture(M, D, 64, 32)
    T = synth.targets(M, K, seed=33)
    d = db(X, metric, "bf16")
    xt = dev(X).requires_grad_(True)
    qt = dev(Q).requires_grad_(True)
    val, idx = knn_topk(qt, xt, d, K, L=L, rerank=2)
    gpu_loss(val, dev(T)).backward()
    V, A = oracle.partial_reduce(oracle.bf16_round(Q), oracle.bf16_round(X), L, metric)
    _, cand = oracle.topk_pairs(V, A, 2 * K)
    ov, oi = oracle.rerank(Q, X, cand, K, metric)
    gi = host(idx).astype(np.int64)
    same = (gi == oi).all(axis=1)
    assert same.mean() > 0.9
    compare_grads(host(qt.grad), host(xt.grad), Q, X, oi, ov, T, metric, same)


def test_autograd_deterministic_and_partial_needs():
    N, M, D, K = 4000, 300, 32, 16
    X = synth.iid_normal(N, D, 41, std=1.0 / np.sqrt(D))
    Q = synth.iid_normal(M, D, 42, std=1.0 / np.sqrt(D))
    T = dev(synth.targets(M, K, seed=43))
    d = db(X, "ip", "bf16")
    grads = []
    for _ in range(2):
        xt = dev(X).requires_grad_(True)
        qt = dev(Q).requires_grad_(True)
        val, _ = knn_topk(qt, xt, d, K, L=256, deterministic=True)
        gpu_loss(val, T).backward()
        grads.append((host(qt.grad), host(xt.grad)))
    assert np.array_equal(grads[0][0], grads[1][0])
    assert np.array_equal(grads[0][1], grads[1][1])
    # only the queries need a gradient: x gets none and the call still works
    qt = dev(Q).requires_grad_(True)
    xt = dev(X)
    val, idx = knn_topk(qt, xt, d, K, L=256, deterministic=True)
    assert not idx.requires_grad
    gpu_loss(val, T).backward()
    assert xt.grad is None
    np.testing.assert_array_equal(host(qt.grad), grads[0][0])


@pytest.mark.parametrize("metric", ["ip", "l2", "cos"])
def test_autograd_directional_finite_differences(metric):
    """d/de loss(Q + eU) and d/de loss(X + eV) by central differences of the
    GPU forward against <dQ, U> and <dX, V>.

    K = N (every row selected) and a loss that weights each selected value by
    a per-row weight w[idx] instead of by rank: softmax is permutation
    equivariant, so the loss is smooth everywhere and re-ordering under the
    perturbation changes nothing."""
    N, M, D = 200, 8, 24
    K = N
    X = synth.iid_normal(N, D, 51, std=1.0 / np.sqrt(D))
    Q = synth.iid_normal(M, D, 52, std=1.0 / np.sqrt(D))
    w = dev(synth.targets(1, N, seed=53)[0]).double()

    def loss_of(val, idx):
        p = torch.softmax(val.double() / TAU, dim=1)
        return (w[idx.long()] * p).sum()

    xt = dev(X).requires_grad_(True)
    qt = dev(Q).requires_grad_(True)
    d = db(X, metric, "f32")
    val, idx = knn_topk(qt, xt, d, K, exact=True)
    loss_of(val, idx).backward()
    gdq, gdx = qt.grad.double(), xt.grad.double()
    g = rng(54)
    eps = 1e-2

    def loss_at(Qn, Xn):
        v, i = knn_topk(dev(Qn), dev(Xn), db(Xn, metric, "f32"), K, exact=True)
        return float(loss_of(v, i))

    for trial in range(3):
        for which in ("q", "x"):
            P = g.standard_normal(Q.shape if which == "q" else X.shape)
            P /= np.linalg.norm(P)
            if which == "q":
                lp, lm = loss_at(Q + eps * P, X), loss_at(Q - eps * P, X)
                an = float((gdq * torch.from_numpy(P).cuda()).sum())
            else:
                lp, lm = loss_at(Q, X + eps * P), loss_at(Q, X - eps * P)
                an = float((gdx * torch.from_numpy(P).cuda()).sum())
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - an) <= 1e-2 * max(abs(an), 0.1), (which, trial, fd, an)


def test_autograd_grad_workload_1m_sampled():
    """N=1M x D=256 BF16 rows N(0,1/D), M=4096, K=32, IP, L from recall 0.95
    rounded to the tile: dQ on sampled queries against the oracle; dX by the
    identities <dX, X> = <dQ, Q> = sum g v (IP) and zero untouched rows."""
    from paper_2206_14286_gb300 import search as S
    w = synth.workload("iid_ip_grad_1m")
    X, Q, K = w["X"], w["Q"], w["K"]
    M, N = Q.shape[0], X.shape[0]
    L = S.plan_bins(N, K, 0.95, round_to=128)
    T = synth.targets(M, K)
    d = db(X, "ip", "bf16")
    xt = dev(X).requires_grad_(True)
    qt = dev(Q).requires_grad_(True)
    val, idx = knn_topk(qt, xt, d, K, L=L, rerank=2)
    vt = val.detach().clone().requires_grad_(True)
    lt = gpu_loss(vt, dev(T))
    lt.backward()
    gv = vt.grad
    val.backward(gv)
    gdq, gdx = qt.grad, xt.grad
    # identities that hold at any size (IP): <dX, X> = sum g v = <dQ, Q>
    s_gv = float((gv.double() * val.detach().double()).sum())
    s_x = float((gdx.double() * xt.detach().double()).sum())
    s_q = float((gdq.double() * qt.detach().double()).sum())
    scale = float((gv.double().abs() * val.detach().double().abs()).sum()) + 1e-30
    assert abs(s_x - s_gv) <= 1e-4 * scale and abs(s_q - s_gv) <= 1e-4 * scale
    touched = torch.zeros(N, dtype=torch.bool, device="cuda")
    touched[idx.reshape(-1).long()] = True
    assert int((gdx[~touched] != 0).sum()) == 0
    # dQ on sampled queries: the oracle's own selection on the BF16 rows
    samp = rng(61).choice(M, size=16, replace=False)
    Vs, As = oracle.partial_reduce(oracle.bf16_round(Q[samp]), oracle.bf16_round(X), L, "ip")
    _, cand = oracle.topk_pairs(Vs, As, 2 * K)
    ov, oi = oracle.rerank(Q[samp], X, cand, K, "ip")
    gi = host(idx)[samp].astype(np.int64)
    same = (gi == oi).all(axis=1)
    assert same.mean() >= 0.75
    g = OL.loss_grad(ov, T[samp], TAU)
    oq, _ = oracle.grad(Q[samp], X, oi, g, "ip", want_dx=False)
    hq = host(gdq)[samp]
    sq = np.abs(oq).max() + 1e-30
    np.testing.assert_allclose(hq[same], oq[same], rtol=0, atol=1e-4 * sq)


@pytest.mark.parametrize("atomic", [False, True])
def test_backward_into_caller_dx_accumulates(atomic):
    """zero_dx=False adds into the caller's dx: two backward passes into one
    buffer give twice one pass (atomic adds of the same values in FP32 may
    round differently, hence the tolerance); zero_dx=True overwrites. Both
    the row kernel and the atomic adds."""
    g = rng(17)
    X = g.standard_normal((5000, 64)).astype(np.float32)
    Q = g.standard_normal((40, 64)).astype(np.float32)
    d = db(X, "ip", "bf16")
    val, idx = d.search(dev(Q), 8, L=128)
    gv = torch.from_numpy(g.standard_normal((40, 8)).astype(np.float32)).cuda()
    _, dx1 = d.backward(dev(Q), idx, gv, want_dq=False, atomic=atomic)
    acc = torch.zeros_like(dx1)
    for _ in range(2):
        d.backward(dev(Q), idx, gv, want_dq=False, dx=acc, zero_dx=False, atomic=atomic)
    torch.cuda.synchronize()
    scale = dx1.abs().max().item()
    assert torch.allclose(acc, 2 * dx1, rtol=0, atol=1e-5 * scale)
    d.backward(dev(Q), idx, gv, want_dq=False, dx=acc, zero_dx=True, atomic=atomic)
    torch.cuda.synchronize()
    assert torch.allclose(acc, dx1, rtol=0, atol=1e-6 * scale)


@pytest.mark.parametrize("metric", ["ip", "l2", "cos"])
def test_deterministic_dense_dx_written_once(metric):
    """deterministic=True with zero_dx: each row of dx is written by one warp,
    zeros or the row's sum in entry order, over whatever dx held (NaN here).
    One row is taken by 600 entries (more than a warp sorts in shared memory),
    some entries are -1 (skipped), K = 37 (two passes of 32 in the dq gather)
    and D = 99 (ragged; the scalar atomic scatter). Checked against the oracle,
    against the zero-then-add ordered path and the atomic path, and
    bit-identical from run to run. Most rows hold more than the 8 entries a
    lane keeps, so both ways of the row kernel run, writing and adding."""
    g = rng(23)
    N, M, D, K = 3000, 600, 99, 37
    X = g.standard_normal((N, D)).astype(np.float32)
    Q = g.standard_normal((M, D)).astype(np.float32)
    idx = g.integers(0, N, size=(M, K)).astype(np.int32)
    idx[:, 0] = 7
    idx[::50, 3] = -1
    gv = g.standard_normal((M, K)).astype(np.float32)
    d = db(X, metric, "bf16")
    xf, Qd, Gd = dev(X), dev(Q), dev(gv)
    Id = torch.from_numpy(idx).cuda()
    outs = []
    for _ in range(2):
        dx = torch.full((N, D), float("nan"), device="cuda")
        dq, _ = d.backward(Qd, Id, Gd, deterministic=True, x_f32=xf, dx=dx, zero_dx=True)
        outs.append((host(dq), host(dx)))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    gdq, gdx = outs[0]
    odq, odx = oracle.grad(Q, X, idx, gv, metric)
    sq, sx = np.abs(odq).max(), np.abs(odx).max()
    np.testing.assert_allclose(gdq, odq, rtol=0, atol=1e-4 * sq)
    np.testing.assert_allclose(gdx, odx, rtol=0, atol=1e-4 * sx)
    touched = np.zeros(N, bool)
    touched[idx[idx >= 0]] = True
    assert not gdx[~touched].any()
    acc = torch.zeros((N, D), device="cuda")
    d.backward(Qd, Id, Gd, want_dq=False, deterministic=True, x_f32=xf, dx=acc, zero_dx=False)
    np.testing.assert_allclose(gdx, host(acc), rtol=0, atol=1e-6 * sx)
    dq_a, dx_a = d.backward(Qd, Id, Gd, x_f32=xf, atomic=True)
    np.testing.assert_array_equal(host(dq_a), gdq)
    np.testing.assert_allclose(host(dx_a), odx, rtol=0, atol=1e-4 * sx)
    # the default (non-deterministic) call takes the same row kernel
    _, dx_d = d.backward(Qd, Id, Gd, x_f32=xf)
    np.testing.assert_array_equal(host(dx_d), gdx)
