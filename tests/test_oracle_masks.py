"""Pins of the mask-pooled oracle (oracle/masks.py): singleton masks reduce it to the per-pixel
iteration of the C oracle; pool and pool_bwd equal the explicit pooling matrix built by loops
and its transpose (hence adjoint); constant regions, empty masks and skipped indices behave as
defined; the pooled loss's gradients match central finite differences through render, pool,
decode and loss."""
import numpy as np
import pytest

import oracle
from oracle import masks as om
from workloads import pixel_masks, random_scene, sam_masks, tiny_scene


def _pool_matrix(offsets, pixels, npix):
    S = len(offsets) - 1
    P = np.zeros((S, npix))
    for m in range(S):
        ids = [int(p) for p in pixels[offsets[m]:offsets[m + 1]] if 0 <= p < npix]
        for p in ids:
            P[m, p] += 1.0 / len(ids)
    return P


def _ragged_csr(rng, npix, S, overlap=True, invalid=True):
    lists = []
    for m in range(S):
        k = int(rng.integers(0, 40)) if m % 7 else 0  # every 7th mask empty
        e = rng.integers(0, npix, size=k)
        if invalid and k and m % 3 == 0:
            e = np.concatenate([e, [-1, npix, npix + 5]])  # skipped entries
        if not overlap:
            e = np.unique(e)
        lists.append(e)
    offsets = np.zeros(S + 1, np.int64)
    offsets[1:] = np.cumsum([len(x) for x in lists])
    return offsets.astype(np.int32), np.concatenate(lists).astype(np.int32)


def test_pool_and_adjoint_equal_the_explicit_matrix():
    rng = np.random.default_rng(0)
    npix, d, S = 150, 5, 23
    off, pix = _ragged_csr(rng, npix, S)
    P = _pool_matrix(off, pix, npix)
    Q = rng.normal(size=(npix, d))
    G = rng.normal(size=(S, d))
    np.testing.assert_allclose(om.pool(Q, off, pix), P @ Q, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(om.pool_bwd(G, off, pix, npix), P.T @ G, rtol=1e-13, atol=1e-15)
    # adjoint: <pool(Q), G> = <Q, pool_bwd(G)>
    assert (om.pool(Q, off, pix) * G).sum() == pytest.approx((Q * om.pool_bwd(G, off, pix, npix)).sum(), rel=1e-12)


def test_constant_regions_empty_masks_and_skipped_indices():
    rng = np.random.default_rng(1)
    npix, d = 60, 3
    Q = np.repeat(rng.normal(size=(6, d)), 10, axis=0)  # six regions of ten equal rows
    lists = [np.arange(10 * r, 10 * r + 10)[rng.permutation(10)[:1 + r]] for r in range(6)] + [np.array([], int)]
    off = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int32)
    pix = np.concatenate(lists).astype(np.int32)
    Qm = om.pool(Q, off, pix)
    np.testing.assert_allclose(Qm[:6], Q[::10], rtol=4e-16, atol=0)  # mean of equal rows is the row
    assert np.all(Qm[6] == 0.0)
    # out-of-range indices are skipped and not counted
    pix2 = np.concatenate([pix[:3], [-4, npix], pix[3:]]).astype(np.int32)
    off2 = off.copy()
    off2[2:] += 2  # the two extra entries sit in mask 1
    np.testing.assert_array_equal(om.pool(Q, off2, pix2), Qm)
    np.testing.assert_array_equal(om.pool_bwd(Qm, off2, pix2, npix), om.pool_bwd(Qm, off, pix, npix))


def test_singleton_masks_reduce_to_the_per_pixel_iteration():
    s = random_scene(3, n=60, d=8, M=10, D=24, width=18, height=14, log_scale=-2.2, mask_drop=0.2)
    cfg = oracle.LossConfig()
    a = om.iteration_masks(s, pixel_masks(s), cfg)
    b = oracle.iteration(s, cfg)
    np.testing.assert_array_equal(a["Qm"], b["Q"])
    for k in ("cos", "l2", "tr", "total", "n_valid"):
        assert a["loss"][k] == b["loss"][k], k
    for k in ("dK", "dV", "dQ", "df"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_one_whole_image_mask_pools_the_mean_query():
    s = random_scene(4, n=80, d=8, M=10, D=24, width=16, height=12, log_scale=-2.2)
    ms = sam_masks(s, cell=(16, 12))  # one region, one cell
    assert ms.n_masks == 1 and ms.pixels.size == s.camera.n_pixels
    out = om.iteration_masks(s, ms)
    np.testing.assert_allclose(out["Qm"][0], out["Q"].mean(axis=0), rtol=1e-12, atol=1e-14)
    # every pixel receives the same gradient dQm / npix
    np.testing.assert_allclose(out["dQ"], np.repeat(out["dQm"] / s.camera.n_pixels, s.camera.n_pixels, 0),
                               rtol=1e-14)


def _total(s, ms, cfg, proj, f, K, V):
    Q = oracle.render_frame(proj, f, s.camera)[0]
    Qm = om.pool(Q, ms.offsets, ms.pixels)
    Fh = oracle.decode(Qm, K, V, cfg.c(Q.shape[1]))[2]
    return oracle.loss(Fh, ms.F, ms.valid, V, s.V0, cfg, Q.shape[1])[0]["total"]


@pytest.mark.parametrize("overlap", [False, True])
def test_pooled_gradients_match_central_differences(overlap):
    s = random_scene(5, n=50, d=4, M=6, D=12, width=20, height=16, log_scale=-2.2)
    ms = sam_masks(s, cell=(5, 4), overlap=overlap, drop=0.2, seed=3, shuffle=True)
    cfg = oracle.LossConfig()
    proj = oracle.project_scene(s)
    out = om.iteration_masks(s, ms, cfg)
    f0, K0, V0 = (x.astype(np.float64) for x in (s.f, s.K, s.V))
    rng = np.random.default_rng(9)
    touched = np.nonzero(np.abs(out["df"]).sum(1) > 0)[0]
    assert len(touched) >= 4
    checks = [("f", (int(g), int(rng.integers(0, s.d)))) for g in touched[:6]]
    checks += [("K", (int(rng.integers(0, s.M)), int(rng.integers(0, s.d)))) for _ in range(5)]
    checks += [("V", (int(rng.integers(0, s.M)), int(rng.integers(0, s.D)))) for _ in range(5)]
    grads = dict(f=out["df"], K=out["dK"], V=out["dV"])
    for name, ix in checks:
        h = 1e-6
        args = dict(f=f0, K=K0, V=V0)
        p, m = args[name].copy(), args[name].copy()
        p[ix] += h
        m[ix] -= h
        ap, am = dict(args, **{name: p}), dict(args, **{name: m})
        num = (_total(s, ms, cfg, proj, **ap) - _total(s, ms, cfg, proj, **am)) / (2 * h)
        assert num == pytest.approx(grads[name][ix], rel=2e-5, abs=1e-9), (name, ix)


def test_mask_sets_partition_and_overlap():
    s = tiny_scene(0)
    npix = s.camera.n_pixels
    a = sam_masks(s, cell=(16, 16))
    cnt = np.bincount(a.pixels, minlength=npix)
    assert np.all(cnt == 1)  # every pixel of a labelled region in exactly one cell mask
    b = sam_masks(s, cell=(16, 16), overlap=True)
    assert np.all(np.bincount(b.pixels, minlength=npix) == 2)
    norms = np.linalg.norm(b.F, axis=1)
    np.testing.assert_allclose(norms, 1.0, rtol=1e-6)


def test_batch_of_pixel_masks_is_the_per_pixel_batch_and_one_frame_is_the_single_step():
    from workloads import room_views
    views = room_views(2, n_views=2, n=4000, width=24, height=18, fx=19.7)
    cfg = oracle.LossConfig()
    a = om.iteration_batch_masks(views, [pixel_masks(v) for v in views], cfg)
    b = oracle.iteration_batch(views, cfg)
    for k in ("cos", "l2", "tr", "total", "n_valid"):
        assert a["loss"][k] == b["loss"][k], k
    np.testing.assert_array_equal(a["dK"], b["dK"])
    np.testing.assert_array_equal(a["dV"], b["dV"])
    np.testing.assert_array_equal(a["df"][id(views[0].f)], b["df"][id(views[0].f)])
    ms = sam_masks(views[0], cell=(6, 6), overlap=True, seed=1)
    c = om.iteration_batch_masks(views[:1], [ms], cfg)
    e = om.iteration_masks(views[0], ms, cfg)
    assert c["loss"]["total"] == e["loss"]["total"]
    np.testing.assert_array_equal(c["df"][id(views[0].f)], e["df"])
