"""FP64 oracle of the streaming K-means dictionary update (Algorithm 1, Eq. stream_kmeans_init,
Sec. III-C "Dictionary Initialization from Streaming Data"): D_t^(0) = StreamKMeans(F_t,
D_{t-1}, K).

TEST INFRASTRUCTURE ONLY (imported by tests/ and never by the product path).

The paper states the procedure in one sentence: the new embeddings are summarised into a few
micro-clusters by a local K-means, which are then merged with the existing global centres and
re-clustered to the fixed dictionary size K (after O'Callaghan et al.'s streaming K-means).
Readings, where it is silent:
  * "micro-factors (5 by default)": the local K-means makes k_micro = 5 micro-clusters per
    keyframe (an explicit argument); the caller draws their initial rows (distinct valid rows
    of F_t) and passes them in;
  * every global centre carries a weight, the number of embeddings it summarises; weight 0
    marks an empty slot.  Slots keep their identity (row j of the dictionary stays row j, so
    its key and its optimiser moments stay attached);
  * merge: the weighted points are the used slots (in slot order) followed by the non-empty
    micro-centres (in micro order); the empty slots, in slot order, take the micro-centres in
    order of decreasing weight (ties: lower micro index) as their initial centres;
  * re-cluster: weighted Lloyd iterations over those points against the centres of the
    occupied slots; a centre becomes the weighted mean of its points and its weight their
    total weight; a centre left without points keeps its position and gets weight 0 (its slot
    is free for the next keyframe);
  * Lloyd: squared Euclidean distance, ties to the lower index, a fixed number of iterations
    (no convergence test), the final weights those of the last assignment; a row flagged
    invalid takes no part.

Parity status: pinned by tests/test_oracle_kmeans.py (a brute-force search of the optimal
partition on tiny inputs reached by Lloyd from a good start; fixed points; well-separated
clusters recovered exactly; the fill and merge rules on hand-built cases; invariance of the
total weight; slot stability).
"""
from __future__ import annotations

import numpy as np


def sq_dist(X, C) -> np.ndarray:
    """||x_i - c_j||^2 for every row pair (the direct definition, a block of rows at a time)."""
    X = np.asarray(X, np.float64)
    C = np.asarray(C, np.float64)
    out = np.empty((X.shape[0], C.shape[0]))
    step = max(1, (1 << 22) // max(1, C.shape[0] * C.shape[1]))
    for i in range(0, X.shape[0], step):
        diff = X[i:i + step, None, :] - C[None, :, :]
        out[i:i + step] = (diff * diff).sum(axis=2)
    return out


def assign(X, C, active=None):
    """Index of the nearest active centre of each row (ties: lowest index) and the gap between
    the second-nearest and the nearest squared distance (inf with one candidate)."""
    dist = sq_dist(X, C)
    if active is not None:
        dist[:, ~np.asarray(active, bool)] = np.inf
    a = np.argmin(dist, axis=1)  # first minimum
    srt = np.sort(dist, axis=1)
    gap = srt[:, 1] - srt[:, 0] if dist.shape[1] > 1 else np.full(dist.shape[0], np.inf)
    return a, gap


def weighted_lloyd(X, w, C0, active, iters: int):
    """`iters` weighted Lloyd iterations from the centres C0 (only `active` ones compete).
    Returns (centres, weights, assignment of the last iteration, smallest decision gap)."""
    X = np.asarray(X, np.float64)
    w = np.asarray(w, np.float64)
    C = np.array(C0, np.float64, copy=True)
    active = np.asarray(active, bool)
    W = np.zeros(C.shape[0])
    a = np.zeros(X.shape[0], np.int64)
    min_gap = np.inf
    for _ in range(iters):
        if X.shape[0] == 0 or not active.any():
            break
        a, gap = assign(X, C, active)
        min_gap = min(min_gap, float(gap.min()))
        for c in np.flatnonzero(active):
            members = a == c
            W[c] = w[members].sum()
            if W[c] > 0:
                C[c] = (w[members, None] * X[members]).sum(axis=0) / W[c]
    return C, W, a, min_gap


def local_kmeans(F, valid, init_idx, iters: int):
    """Micro-clusters of the valid rows of F: centres (k x D), weights (row counts), the
    assignment of every row (-1 for invalid rows) and the smallest decision gap."""
    F = np.asarray(F, np.float64)
    n = F.shape[0]
    valid = np.ones(n, bool) if valid is None else np.asarray(valid).astype(bool)
    rows = np.flatnonzero(valid)
    init_idx = np.asarray(init_idx, np.int64)
    C0 = F[init_idx]
    C, W, a, gap = weighted_lloyd(F[rows], np.ones(rows.size), C0, np.ones(len(init_idx), bool), iters)
    full = np.full(n, -1, np.int64)
    if iters > 0:
        full[rows] = a
    return C, W, full, gap


def merge_and_recluster(C_prev, w_prev, micro_C, micro_w, iters: int):
    """The merge and re-clustering of the global step.  Returns (centres, weights, the points'
    assignment, smallest decision gap)."""
    C_prev = np.asarray(C_prev, np.float64)
    w_prev = np.asarray(w_prev, np.float64)
    micro_C = np.asarray(micro_C, np.float64)
    micro_w = np.asarray(micro_w, np.float64)
    K = C_prev.shape[0]
    used = np.flatnonzero(w_prev > 0)
    live = np.flatnonzero(micro_w > 0)
    P = np.concatenate([C_prev[used], micro_C[live]])
    pw = np.concatenate([w_prev[used], micro_w[live]])
    C0 = C_prev.copy()
    active = w_prev > 0
    # empty slots take the heaviest micro-centres first (stable: ties by micro index)
    order = sorted(live.tolist(), key=lambda c: (-micro_w[c], c))
    empty = np.flatnonzero(w_prev <= 0)
    for slot, c in zip(empty, order):
        C0[slot] = micro_C[c]
        active[slot] = True
    C, W, a, gap = weighted_lloyd(P, pw, C0, active, iters)
    return C, W, a, gap


def stream_kmeans(F, valid, C_prev, w_prev, init_idx, iters_local: int = 10, iters_global: int = 10) -> dict:
    """StreamKMeans(F_t, D_{t-1}, K): the new centres D_t^(0) (K x D) and weights, with the
    micro-clusters and the smallest decision gap of both Lloyd phases (iteration counts >= 1)."""
    assert iters_local >= 1 and iters_global >= 1
    mC, mW, ma, g1 = local_kmeans(F, valid, init_idx, iters_local)
    C, W, pa, g2 = merge_and_recluster(C_prev, w_prev, mC, mW, iters_global)
    return dict(centres=C, weights=W, micro_centres=mC, micro_weights=mW, micro_assign=ma,
                min_gap=min(g1, g2))
