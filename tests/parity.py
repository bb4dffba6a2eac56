"""Comparison rules between the CUDA path and the FP64 oracle.

A query is *decided* when every score margin that fixes the answer exceeds
twice the tolerance (both sides may err by one tolerance):
  * bin-wise step (scores of the stored, possibly low-precision rows): the
    gap between the Kp-th and (Kp+1)-th bin winners, and the gap between the
    best and second-best row of every bin whose winner is among the best
    Kp+1;
  * final step (FP32-row scores of the oracle's Kp candidates): the gap
    between the K-th and (K+1)-th candidate (if Kp > K) and between adjacent
    ranks of the first K.
Decided queries must return the oracle's indices exactly. Undecided queries
must return, at every rank, a value within tolerance of the oracle's value at
that rank, and indices whose own oracle score matches the returned value and
which are within tolerance of their bin's best.

Tolerances are relative to the natural scale of a score: ||q|| max||x|| for
IP/COS, ||q||^2 + max||x||^2 for L2.
"""
import numpy as np

REL_F32 = 1e-5
REL_LOWP = 1e-2


def score_matrix(Q, X, metric, chunk=1 << 14):
    """FP64 larger-is-better scores: IP <q,x>, L2 -||q-x||^2, COS cosine."""
    Q = np.asarray(Q, np.float64)
    M, N = Q.shape[0], X.shape[0]
    out = np.empty((M, N), np.float64)
    qn2 = (Q * Q).sum(1)
    for s in range(0, N, chunk):
        Xc = np.asarray(X[s:s + chunk], np.float64)
        G = Q @ Xc.T
        if metric == "ip":
            out[:, s:s + chunk] = G
        elif metric == "l2":
            xn2 = (Xc * Xc).sum(1)
            out[:, s:s + chunk] = -(qn2[:, None] + xn2[None, :] - 2.0 * G)
        else:
            xn = np.sqrt((Xc * Xc).sum(1))
            qn = np.sqrt(qn2)
            with np.errstate(invalid="ignore", divide="ignore"):
                c = G / (qn[:, None] * xn[None, :])
            out[:, s:s + chunk] = np.nan_to_num(c)
    return out


def query_scale(Q, X, metric):
    Q = np.asarray(Q, np.float64)
    qn2 = (Q * Q).sum(1)
    xmax2 = float(max((np.asarray(X[s:s + 65536], np.float64) ** 2).sum(1).max()
                      for s in range(0, X.shape[0], 65536)))
    if metric == "l2":
        return qn2 + xmax2
    if metric == "cos":
        return np.ones_like(qn2)
    return np.sqrt(qn2 * xmax2)


def reported(S, metric):
    return -S if metric == "l2" else S


def bin_best_second(S, L, bins="mod"):
    M, N = S.shape
    if bins == "contiguous":
        best = np.empty((M, L))
        second = np.full((M, L), -np.inf)
        for b, rows in enumerate(np.array_split(np.arange(N), L)):
            blk = S[:, rows]
            if rows.size >= 2:
                part = -np.partition(-blk, 1, axis=1)
                best[:, b], second[:, b] = part[:, 0], part[:, 1]
            else:
                best[:, b] = blk[:, 0]
        return best, second
    nb = -(-N // L)
    P = np.full((M, nb * L), -np.inf)
    P[:, :N] = S
    P = P.reshape(M, nb, L)
    if nb >= 2:
        part = -np.partition(-P, 1, axis=1)
        return part[:, 0, :], part[:, 1, :]
    return P[:, 0, :], np.full((M, L), -np.inf)


def decided_mask(S_lp, L, Kp, S_f, cand, K, tol, tol_final=None, bins="mod"):
    """Boolean per query; cand = the oracle's Kp candidates (M x Kp).
    tol applies to the bin step, tol_final (default tol) to the FP32 order."""
    best, second = bin_best_second(S_lp, L, bins)
    sc = np.take_along_axis(S_f, np.maximum(cand, 0), 1)
    sc = np.where(cand >= 0, sc, -np.inf)
    return decided_from_stats(best, second, Kp, sc, K, tol, tol_final)


def decided_from_stats(best, second, Kp, cand_f, K, tol, tol_final=None):
    """decided_mask from per-bin statistics: best / second are the largest and
    second-largest low-precision score of every bin (M x L), cand_f the FP32
    scores of the oracle's Kp candidates (M x Kp, -inf for none)."""
    if tol_final is None:
        tol_final = tol
    M, L = best.shape
    ok = np.ones(M, bool)
    w = -np.sort(-best, axis=1)
    if L > Kp:
        ok &= (w[:, Kp - 1] - w[:, Kp]) > 2 * tol
    thr = w[:, min(Kp, L - 1)]
    relevant = best >= thr[:, None]
    ok &= np.all(~relevant | ((best - second) > 2 * tol[:, None]), axis=1)
    sc = -np.sort(-np.asarray(cand_f, np.float64), axis=1)
    upto = min(K + 1, Kp) if Kp > K else K
    if upto >= 2:
        gaps = sc[:, :upto - 1] - sc[:, 1:upto]
        ok &= np.all(gaps > 2 * tol_final[:, None], axis=1)
    return ok


def bin_best_second_chunked(score_rows, N, L, chunk):
    """bin_best_second (bins j mod L) over row chunks: score_rows(c0, c1)
    returns the M x (c1 - c0) scores of rows c0..c1-1. chunk must be a
    multiple of L, so a row keeps its bin inside its chunk; the maxima of the
    chunks merge into the best and second best of each bin."""
    assert chunk % L == 0
    best = second = None
    for c0 in range(0, N, chunk):
        b, s = bin_best_second(score_rows(c0, min(N, c0 + chunk)), L)
        if best is None:
            best, second = b, s
        else:
            best, second = (np.maximum(best, b),
                            np.maximum(np.maximum(second, s), np.minimum(best, b)))
    return best, second


def bin_of_rows(N, L, bins):
    if bins == "contiguous":
        return np.concatenate([np.full(len(r), b) for b, r in
                               enumerate(np.array_split(np.arange(N), L))])
    return np.arange(N) % L


def check_search(gpu_val, gpu_idx, orc_val, orc_idx, S_lp, S_f, L, metric, tol, decided,
                 bins="mod"):
    """Asserts the rules above; returns the fraction of decided queries."""
    best, _ = bin_best_second(S_lp, L, bins)
    owner = bin_of_rows(S_lp.shape[1], L, bins)
    return check_search_core(gpu_val, gpu_idx, orc_val, orc_idx,
                             lambda i, j: S_lp[i, j], lambda i, j: S_f[i, j],
                             best, lambda j: owner[j], metric, tol, decided)


def check_search_core(gpu_val, gpu_idx, orc_val, orc_idx, lp_at, f_at, best, owner_of, metric,
                      tol, decided):
    """check_search without the full score matrices: lp_at(i, j) / f_at(i, j)
    give query i's low-precision / FP32-row scores of the rows j, best is the
    M x L array of bin maxima and owner_of(j) the bins of rows j."""
    gpu_val = np.asarray(gpu_val, np.float64)
    gpu_idx = np.asarray(gpu_idx, np.int64)
    M, K = gpu_idx.shape
    bad = []
    for i in range(M):
        if decided[i]:
            if not np.array_equal(gpu_idx[i], orc_idx[i]):
                bad.append((i, "idx", gpu_idx[i][:8], orc_idx[i][:8]))
                continue
        if np.any(np.abs(gpu_val[i] - orc_val[i]) > tol[i]):
            bad.append((i, "val-by-rank", gpu_val[i][:6], orc_val[i][:6]))
            continue
        j = gpu_idx[i]
        if np.any(j < 0) or len(set(j.tolist())) != K:
            bad.append((i, "invalid idx", j[:8]))
            continue
        own = reported(np.asarray(f_at(i, j), np.float64), metric)
        if np.any(np.abs(own - gpu_val[i]) > tol[i]):
            bad.append((i, "own value", own[:6], gpu_val[i][:6]))
            continue
        if np.any(np.asarray(lp_at(i, j), np.float64) < best[i, owner_of(j)] - tol[i]):
            bad.append((i, "not a bin maximum", j[:8]))
    assert not bad, "%d of %d queries disagree, e.g. %s" % (len(bad), M, bad[:3])
    return float(np.mean(decided))


def fp32_acc_tol(Qs, Xs, metric):
    """Per query: the bin-step tolerance of the BF16 tensor-core contraction,
    which keeps the FP32 accumulator in its keys. FP32 accumulation of D exact
    BF16 products errs by about D u ||q|| ||x|| at worst (u = 2^-24), well
    inside 3e-5 of the natural scale for D <= 4096 in practice; for L2 the half
    norm enters as a three-part BF16 split, within 2^-24 of it, and the
    larger-is-better score -||q-x||^2 doubles both."""
    t = 3e-5 * query_scale(Qs, Xs, metric)
    if metric == "l2":
        xmax2 = float(max((np.asarray(Xs[s:s + 65536], np.float64) ** 2).sum(1).max()
                          for s in range(0, Xs.shape[0], 65536)))
        t = t + 2.0 ** -20 * xmax2
    return t
