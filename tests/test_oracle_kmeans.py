"""Pins of the streaming K-means oracle (oracle/kmeans.py): Lloyd against scipy's kmeans2 from
the same start, a brute-force optimal partition of tiny inputs as a fixed point, monotone
objective, exact recovery of well-separated clusters, weighted means, the fill and merge rules
of the global step on hand-built dictionaries, conservation of the total weight, slot
stability and the exclusion of invalid rows."""
import itertools

import numpy as np
import pytest

from oracle import kmeans as km


def _sse(X, w, C, a):
    return float((w * ((X - C[a]) ** 2).sum(1)).sum())


def test_local_lloyd_matches_scipy_kmeans2():
    vq = pytest.importorskip("scipy.cluster.vq")
    rng = np.random.default_rng(0)
    X = rng.normal(size=(300, 6))
    init = rng.choice(300, size=5, replace=False)
    C, W, a, _ = km.local_kmeans(X, None, init, 7)
    Cs, _ = vq.kmeans2(X, X[init].copy(), iter=7, minit="matrix", missing="warn")
    np.testing.assert_allclose(C, Cs, rtol=1e-12, atol=1e-12)
    assert W.sum() == 300 and np.all(np.bincount(a, minlength=5) == W)


def test_optimal_partition_is_a_fixed_point_and_objective_decreases():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(8, 2))
    w = rng.uniform(0.5, 3.0, size=8)
    best, best_lab = np.inf, None
    for lab in itertools.product(range(3), repeat=8):  # brute force over all 3-partitions
        lab = np.array(lab)
        if len(set(lab)) < 3:
            continue
        C = np.array([np.average(X[lab == c], axis=0, weights=w[lab == c]) for c in range(3)])
        e = _sse(X, w, C, lab)
        if e < best:
            best, best_lab = e, lab
    C0 = np.array([np.average(X[best_lab == c], axis=0, weights=w[best_lab == c]) for c in range(3)])
    C, W, a, _ = km.weighted_lloyd(X, w, C0, np.ones(3, bool), 5)
    np.testing.assert_allclose(C, C0, rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(a, best_lab)
    assert _sse(X, w, C, a) == pytest.approx(best)
    # from a poor start the weighted objective never increases
    C1 = X[:3].copy()
    prev = np.inf
    for it in range(1, 7):
        C, W, a, _ = km.weighted_lloyd(X, w, C1, np.ones(3, bool), it)
        e = _sse(X, w, C, km.assign(X, C)[0])
        assert e <= prev + 1e-12
        prev = e


def test_well_separated_clusters_are_recovered():
    rng = np.random.default_rng(2)
    centres = rng.normal(size=(5, 16)) * 10
    lab = rng.integers(0, 5, size=400)
    X = centres[lab] + rng.normal(size=(400, 16)) * 0.05
    init = [int(np.flatnonzero(lab == c)[0]) for c in range(5)]
    C, W, a, gap = km.local_kmeans(X, None, init, 3)
    np.testing.assert_array_equal(a, lab)
    for c in range(5):
        np.testing.assert_allclose(C[c], X[lab == c].mean(0), rtol=1e-12)
        assert W[c] == (lab == c).sum()
    assert gap > 1.0


def test_fill_rule_on_an_empty_dictionary():
    rng = np.random.default_rng(3)
    Cp = rng.normal(size=(6, 4))
    mC = rng.normal(size=(3, 4)) * 5
    mW = np.array([2.0, 7.0, 2.0])
    C, W, _, _ = km.merge_and_recluster(Cp, np.zeros(6), mC, mW, 3)
    # slots 0, 1, 2 take micro 1 (heaviest), then 0 and 2 (equal weights, lower index first)
    np.testing.assert_array_equal(C[:3], mC[[1, 0, 2]])
    np.testing.assert_array_equal(W, [7.0, 2.0, 2.0, 0.0, 0.0, 0.0])
    np.testing.assert_array_equal(C[3:], Cp[3:])


def test_merge_into_a_full_dictionary_conserves_weight_and_slots():
    rng = np.random.default_rng(4)
    Cp = rng.normal(size=(5, 8)) * 10  # far apart
    wp = np.array([3.0, 1.0, 4.0, 1.0, 5.0])
    mC = np.stack([Cp[2] + 0.01, Cp[0]])  # near slot 2, on slot 0
    mW = np.array([4.0, 2.0])
    C, W, a, gap = km.merge_and_recluster(Cp, wp, mC, mW, 4)
    assert W.sum() == wp.sum() + mW.sum()
    np.testing.assert_array_equal(W, [5.0, 1.0, 8.0, 1.0, 5.0])
    np.testing.assert_allclose(C[2], (4 * Cp[2] + 4 * mC[0]) / 8, rtol=1e-12)
    np.testing.assert_allclose(C[0], Cp[0], rtol=1e-12)
    np.testing.assert_allclose(C[[1, 3, 4]], Cp[[1, 3, 4]], rtol=1e-15)  # untouched slots do not move
    assert gap > 1.0


def test_partly_filled_dictionary_and_invalid_rows():
    rng = np.random.default_rng(5)
    F = rng.normal(size=(60, 10))
    valid = (rng.uniform(size=60) > 0.3).astype(np.uint8)
    rows = np.flatnonzero(valid)
    init = rows[[0, 5, 9]]
    Cp = rng.normal(size=(8, 10))
    wp = np.array([2.0, 0, 3.0, 0, 0, 1.0, 0, 0])
    r = km.stream_kmeans(F, valid, Cp, wp, init, 6, 6)
    # the invalid rows take no part: the same as clustering the compacted rows
    r2 = km.stream_kmeans(F[rows], None, Cp, wp, [0, 5, 9], 6, 6)
    np.testing.assert_allclose(r["centres"], r2["centres"], rtol=1e-13)
    np.testing.assert_array_equal(r["weights"], r2["weights"])
    assert np.all(r["micro_assign"][valid == 0] == -1)
    assert r["weights"].sum() == wp.sum() + valid.sum()
