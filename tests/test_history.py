"""The history buffer's sampler (Algorithm 1, Sec. III-C): B distinct keyframes, uniform over
the stored ones, all of them when fewer than B are stored, reproducible from its seed."""
import itertools

import numpy as np
import pytest

from paper_2602_12314_gb300.history import KeyframeHistory


def test_sample_sizes_and_distinctness():
    h = KeyframeHistory(0)
    assert h.sample(3) == [] and h.batch("new", 3) == ["new"]
    for i in range(5):
        h.add(i)
    assert sorted(h.sample(10)) == [0, 1, 2, 3, 4]
    for _ in range(50):
        s = h.sample(3)
        assert len(s) == 3 and len(set(s)) == 3
    assert h.sample(0) == []
    with pytest.raises(ValueError):
        h.sample(-1)
    b = h.batch("new", 2)
    assert b[0] == "new" and len(b) == 3


def test_subsets_are_uniform():
    h = KeyframeHistory(7)
    for i in range(5):
        h.add(i)
    trials = 20000
    counts = {c: 0 for c in itertools.combinations(range(5), 2)}
    for _ in range(trials):
        counts[tuple(sorted(h.sample(2)))] += 1
    expected = trials / len(counts)
    chi2 = sum((c - expected) ** 2 / expected for c in counts.values())
    assert chi2 < 27.9  # chi-square, 9 degrees of freedom, p = 0.001


def test_seeded_reproducibility():
    a, b = KeyframeHistory(3), KeyframeHistory(3)
    for i in range(9):
        a.add(i)
        b.add(i)
    assert [a.sample(4) for _ in range(5)] == [b.sample(4) for _ in range(5)]
