"""The history buffer of Algorithm 1 (Sec. III-C, historical learning against catastrophic
forgetting): the keyframes mapped so far, from which B are drawn uniformly at random, without
replacement, to join each new keyframe's optimisation batch.  Host logic only."""
from __future__ import annotations

import numpy as np


class KeyframeHistory:
    """Append-only list of keyframes with a seeded uniform sampler."""

    def __init__(self, seed: int = 0):
        self._items: list = []
        self._rng = np.random.default_rng(seed)

    def __len__(self) -> int:
        return len(self._items)

    def __getitem__(self, i):
        return self._items[i]

    def add(self, keyframe) -> None:
        """Algorithm 1's last step: the keyframe joins the history after its optimisation."""
        self._items.append(keyframe)

    def sample(self, B: int) -> list:
        """B distinct keyframes drawn uniformly (all of them, in a random order, when fewer
        than B are stored); each subset of size B is equally likely."""
        if B < 0:
            raise ValueError("B must be >= 0")
        k = min(B, len(self._items))
        if k == 0:
            return []
        idx = self._rng.choice(len(self._items), size=k, replace=False)
        return [self._items[i] for i in idx]

    def batch(self, new_keyframe, B: int) -> list:
        """The training batch of Algorithm 1: the new keyframe followed by B sampled ones."""
        return [new_keyframe] + self.sample(B)
