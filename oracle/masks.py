"""FP64 oracle of the mask-pooled form of the step: one query and one target per SAM mask
instead of one per pixel (Sec. III-B, Eq. render_query: with SAM-based targets, n is the
number of valid masks and each target is pooled over its mask's region).

TEST INFRASTRUCTURE ONLY (imported by tests/, the smoke check and the bench's CPU legs; never
by the product path).

Readings of the paper (it states only that n counts the masks and that the targets are
mask-pooled):
  * the query of mask m is the mean of the rendered per-pixel queries over the mask's
    pixels, Qm_m = (1/|m|) sum_{p in m} Q_p, the same pooling the targets get;
  * masks are lists of pixel indices (row = y * W + x) and may overlap (SAM returns masks of
    several granularities); a pixel index outside [0, H*W) is skipped and not counted, and
    an empty mask pools to the zero vector;
  * the decode, the loss and the trust region are those of the per-pixel step with the rows
    of Qm and the per-mask targets in place of the pixels; the loss set is the caller's
    per-mask flags.

The backward of the pooling is its adjoint: dQ_p = sum_{m containing p} dQm_m / |m|.  The
pooled iteration composes the untiled renderer, the decode, the loss and the analytic
backward of the C oracle with the two functions below.

Parity status: pinned by tests/test_oracle_masks.py (singleton masks reduce to the per-pixel
iteration; the adjoint identity of pool / pool_bwd; pooling of constant regions; skipped
indices; central finite differences of the pooled loss with respect to f, K, V).
"""
from __future__ import annotations

import numpy as np


def mask_entries(offsets, pixels, npix: int, m: int) -> np.ndarray:
    """The valid pixel indices of mask m (its CSR entries that lie in [0, npix))."""
    e = np.asarray(pixels[int(offsets[m]):int(offsets[m + 1])], np.int64)
    return e[(e >= 0) & (e < npix)]


def pool(Q, offsets, pixels) -> np.ndarray:
    """Qm (S x d): the mean of the rows of Q over each mask; zero for an empty mask."""
    Q = np.asarray(Q, np.float64)
    npix, d = Q.shape
    S = len(offsets) - 1
    Qm = np.zeros((S, d))
    for m in range(S):
        e = mask_entries(offsets, pixels, npix, m)
        if e.size:
            Qm[m] = Q[e].sum(axis=0) / e.size
    return Qm


def pool_bwd(dQm, offsets, pixels, npix: int) -> np.ndarray:
    """dQ (npix x d): each mask hands dQm_m / |m| to every one of its pixels (summed where
    masks overlap, and over repeated indices of one mask)."""
    dQm = np.asarray(dQm, np.float64)
    S, d = dQm.shape
    dQ = np.zeros((npix, d))
    for m in range(S):
        e = mask_entries(offsets, pixels, npix, m)
        if e.size:
            np.add.at(dQ, e, dQm[m] / e.size)  # unbuffered: a repeated index adds once per entry
    return dQ


def iteration_masks(scene, masks, cfg=None, f=None, K=None, V=None, with_df=True) -> dict:
    """One forward + backward of the mask-pooled step (no optimiser update): render ->
    pool -> decode -> loss over the masks -> dQm, dK, dV -> dQ (pool adjoint) -> df.
    `masks` carries offsets, pixels, the per-mask targets F (S x D) and flags valid (S,)."""
    import oracle

    cfg = cfg or oracle.LossConfig()
    f = scene.f if f is None else f
    K = scene.K if K is None else K
    V = scene.V if V is None else V
    proj = oracle.project_scene(scene)
    Q = oracle.render_frame(proj, f, scene.camera)[0]
    Qm = pool(Q, masks.offsets, masks.pixels)
    _, A, Fh = oracle.decode(Qm, K, V, cfg.c(Q.shape[1]))
    parts, cos_p = oracle.loss(Fh, masks.F, masks.valid, V, scene.V0, cfg, Q.shape[1])
    dQm, dK, dV = oracle.backward(Qm, K, V, scene.V0, A, Fh, masks.F, masks.valid, cfg)
    dQ = pool_bwd(dQm, masks.offsets, masks.pixels, Q.shape[0])
    out = dict(Q=Q, Qm=Qm, A=A, Fhat=Fh, loss=parts, cos_p=cos_p, dQm=dQm, dQ=dQ, dK=dK, dV=dV)
    if with_df:
        out["df"] = oracle.render_frame_bwd(proj, dQ, scene.camera, np.asarray(f).shape[0], Q.shape[1])
    return out


def iteration_batch_masks(scenes, mask_sets, cfg=None) -> dict:
    """One forward + backward over a batch of keyframes sharing the dictionary, mask-pooled:
    every frame rendered untiled and pooled over its own masks, the pooled rows, targets and
    flags stacked in frame order, one decode / loss / backward over the stack (one trust-region
    term), the query gradients pooled back to each frame's pixels and rendered back; df summed
    over the frames that render the same query array (grouped by the identity of f)."""
    import oracle

    cfg = cfg or oracle.LossConfig()
    s0 = scenes[0]
    projs = [oracle.project_scene(s) for s in scenes]
    Qs = [oracle.render_frame(p, s.f, s.camera)[0] for p, s in zip(projs, scenes)]
    Qm = np.concatenate([pool(Q, ms.offsets, ms.pixels) for Q, ms in zip(Qs, mask_sets)])
    F = np.concatenate([ms.F for ms in mask_sets])
    valid = np.concatenate([ms.valid for ms in mask_sets])
    _, A, Fh = oracle.decode(Qm, s0.K, s0.V, cfg.c(Qm.shape[1]))
    parts, _ = oracle.loss(Fh, F, valid, s0.V, s0.V0, cfg, Qm.shape[1])
    dQm, dK, dV = oracle.backward(Qm, s0.K, s0.V, s0.V0, A, Fh, F, valid, cfg)
    df = {}
    row = 0
    for p, s, ms in zip(projs, scenes, mask_sets):
        S = ms.n_masks
        dQ = pool_bwd(dQm[row:row + S], ms.offsets, ms.pixels, s.camera.n_pixels)
        g = oracle.render_frame_bwd(p, dQ, s.camera, s.n, Qm.shape[1])
        df[id(s.f)] = df.get(id(s.f), 0.0) + g
        row += S
    return dict(Qm=Qm, loss=parts, dK=dK, dV=dV, dQm=dQm, df=df)

