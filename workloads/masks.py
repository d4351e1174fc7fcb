"""Seeded SAM-style mask sets for the mask-pooled step (no method arithmetic beyond building
the inputs): masks are the scene's surface regions cut into image cells (the
over-segmentation an automatic SAM mask generator gives on walls and floors), optionally
with the whole regions added as coarser masks that overlap the cells (SAM's several
granularities).  Each mask's target is the l2-normalised mean of the scene's per-pixel
targets over the mask, standing in for mask-pooled normalised CLIP/DINO embeddings."""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class MaskSet:
    offsets: np.ndarray  # (S+1,) int32 CSR offsets into pixels
    pixels: np.ndarray   # (E,) int32 pixel indices, row = y*W + x
    F: np.ndarray        # (S, D) float32 per-mask targets
    valid: np.ndarray    # (S,) uint8, 1 = mask in the loss set

    @property
    def n_masks(self) -> int:
        return self.offsets.shape[0] - 1


def _csr(lists):
    offsets = np.zeros(len(lists) + 1, np.int64)
    offsets[1:] = np.cumsum([len(x) for x in lists])
    pixels = np.concatenate(lists) if lists else np.zeros(0, np.int64)
    return offsets.astype(np.int32), pixels.astype(np.int32)


def _targets(F, lists):
    out = np.zeros((len(lists), F.shape[1]))
    for m, e in enumerate(lists):
        if len(e):
            v = F[e].astype(np.float64).mean(axis=0)
            out[m] = v / max(np.linalg.norm(v), 1e-12)
    return out.astype(np.float32)


def sam_masks(scene, cell=(80, 60), overlap: bool = False, drop: float = 0.0, seed: int = 0,
              shuffle: bool = False) -> MaskSet:
    """Masks = (region, cell) pairs present in the image (region = scene.labels, or one region
    for a scene without labels; pixels labelled -1 belong to no mask), in order of region then
    cell, each listing its pixels in raster order (shuffled when `shuffle`).  With `overlap`,
    every region is also one whole mask (appended after the cells).  A fraction `drop` of the
    masks is flagged out of the loss set."""
    cam = scene.camera
    W, H = cam.width, cam.height
    lab = scene.labels if scene.labels is not None else np.zeros(W * H, np.int32)
    cw, ch = cell
    ncx = (W + cw - 1) // cw
    yy, xx = np.divmod(np.arange(W * H), W)
    cid = (yy // ch) * ncx + xx // cw
    ncell = ((H + ch - 1) // ch) * ncx
    key = np.where(lab >= 0, lab.astype(np.int64) * ncell + cid, -1)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    start = np.searchsorted(ks, 0)
    ks, order = ks[start:], order[start:]
    cut = np.flatnonzero(np.diff(ks)) + 1
    lists = np.split(order, cut) if ks.size else []
    if overlap:
        lk = lab[order]
        lcut = np.flatnonzero(np.diff(lk)) + 1
        lists += [np.sort(x) for x in np.split(order, lcut)] if ks.size else []
    rng = np.random.default_rng(seed)
    if shuffle:
        lists = [rng.permutation(x) for x in lists]
    offsets, pixels = _csr(lists)
    valid = (rng.uniform(size=len(lists)) >= drop).astype(np.uint8)
    return MaskSet(offsets=offsets, pixels=pixels, F=_targets(scene.F, lists), valid=valid)


def pixel_masks(scene) -> MaskSet:
    """Every pixel its own mask, with the scene's per-pixel targets and loss set: the
    mask-pooled step on these masks is the per-pixel step."""
    n = scene.camera.n_pixels
    return MaskSet(offsets=np.arange(n + 1, dtype=np.int32), pixels=np.arange(n, dtype=np.int32),
                   F=np.ascontiguousarray(scene.F, np.float32), valid=np.ascontiguousarray(scene.mask, np.uint8))
