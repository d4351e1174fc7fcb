"""Parity of the mask-pooled path (SAM-based targets: one decoded row and one target per mask)
with the FP64 oracle of oracle/masks.py, through the C ABI.

Pooling: per-mask means within a relative 1e-5 per row (float32 sums of at most a few
thousand rows), its adjoint likewise, bit-identical on repeated calls.  The step: the loss of
the first iteration within 1e-4 (FP32) / 5e-3 (BF16) of the oracle, the Adam update of the
first step (-lr sign(g)) wherever the oracle's gradient is well above rounding, and singleton
masks reproduce the per-pixel step."""
import numpy as np
import pytest

import oracle
from oracle import masks as om
from workloads import pixel_masks, random_scene, room_scene, sam_masks, tiny_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2602_12314_gb300 import api as _api
    return _api


@pytest.fixture(scope="module")
def ctx(api):
    c = api.Context(0)
    yield c
    c.close()


def _dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _csr(rng, npix, S, big=3000):
    """Ragged masks: one of `big` entries (several chunks), empty ones, repeated and skipped
    indices, overlaps, shuffled order."""
    lists = []
    for m in range(S):
        if m == 1:
            k = big
        elif m % 9 == 0:
            k = 0
        else:
            k = int(rng.integers(1, 600))
        e = rng.integers(0, npix, size=k)
        if k and m % 4 == 0:
            e = np.concatenate([e, [-1, npix, -7, npix + 3]])
        lists.append(rng.permutation(e))
    off = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int32)
    return off, np.concatenate(lists).astype(np.int32)


def _rel_rows(a, b, floor=1e-6):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), floor)


@pytest.mark.parametrize("d", [16, 32, 64])
def test_pool_and_adjoint_match_oracle(api, ctx, d):
    rng = np.random.default_rng(d)
    npix, S = 5003, 37
    off, pix = _csr(rng, npix, S)
    Q = rng.normal(size=(npix, d)).astype(np.float32)
    G = rng.normal(size=(S, d)).astype(np.float32)
    Qm = api.pool_queries(ctx, _dev(Q), off, pix).cpu().numpy().astype(np.float64)
    Qo = om.pool(Q, off, pix)
    nonempty = np.abs(Qo).sum(1) > 0
    assert _rel_rows(Qm[nonempty], Qo[nonempty]).max() <= 1e-5
    assert np.all(Qm[~nonempty] == 0.0)
    dQ = api.pool_queries_bwd(ctx, _dev(G), off, pix, npix).cpu().numpy().astype(np.float64)
    dQo = om.pool_bwd(G, off, pix, npix)
    np.testing.assert_allclose(dQ, dQo, rtol=1e-5, atol=1e-6 * np.abs(dQo).max())
    # fixed chunking and summation order: repeated calls are bit-identical
    again = api.pool_queries(ctx, _dev(Q), off, pix).cpu().numpy()
    np.testing.assert_array_equal(again, Qm.astype(np.float32))


def test_pool_degenerate_inputs(api, ctx):
    rng = np.random.default_rng(5)
    Q = _dev(rng.normal(size=(50, 32)))
    # no masks
    assert api.pool_queries(ctx, Q, np.zeros(1, np.int32), np.zeros(0, np.int32)).shape == (0, 32)
    dQ = api.pool_queries_bwd(ctx, torch.zeros((0, 32), device="cuda"), np.zeros(1, np.int32),
                              np.zeros(0, np.int32), 50)
    assert float(dQ.abs().max()) == 0.0
    # masks without entries, a decreasing offset pair and offsets past the end pool to zero
    off = np.array([0, 0, 3, 2, 9, 12], np.int32)
    pix = np.array([4, 5, 6, 7, 8], np.int32)
    Qm = api.pool_queries(ctx, Q, off, pix).cpu().numpy()
    Qo = om.pool(Q.cpu().numpy(), off, pix)
    np.testing.assert_allclose(Qm, Qo, rtol=1e-6, atol=1e-7)
    assert np.all(Qm[[0, 2, 4]] == 0.0)
    # an empty image: every index skipped
    Qe = api.pool_queries(ctx, torch.zeros((0, 16), device="cuda"), np.array([0, 2], np.int32),
                          np.array([0, 1], np.int32))
    assert Qe.shape == (1, 16) and float(Qe.abs().max()) == 0.0


def test_pool_rejects_bad_arguments(api, ctx):
    from paper_2602_12314_gb300 import _lib as L
    Q = torch.zeros((10, 24), device="cuda")
    with pytest.raises(L.LatentamError) as e:
        api.pool_queries(ctx, Q, np.array([0, 1], np.int32), np.array([0], np.int32))
    assert e.value.status == L.ERR_UNSUPPORTED_SHAPE


def _first_update_check(x0, got, g, lr=0.01):
    x = x0.astype(np.float64).copy()
    m, v = np.zeros_like(x), np.zeros_like(x)
    oracle.adam(x.reshape(-1), g.reshape(-1), m.reshape(-1), v.reshape(-1), 1, lr)
    well = np.abs(g) > 1e-2 * np.abs(g).max()
    np.testing.assert_allclose(got[well], x[well], rtol=0, atol=1e-4 * lr + 1e-6)
    assert np.all(np.abs(got - x0) <= lr * 1.0001 + 1e-6)


@pytest.mark.parametrize("overlap", [False, True])
def test_step_one_iteration_matches_oracle(api, ctx, overlap):
    s = tiny_scene(0)
    ms = sam_masks(s, cell=(16, 16), overlap=overlap, drop=0.2, seed=1, shuffle=True)
    st = api.LatentStep(ctx, s, precision=api.FP32, masks=ms)
    loss = st.step(iters=1, learn_f=True)
    o = om.iteration_masks(s, ms, oracle.LossConfig())
    assert loss["n_valid"] == o["loss"]["n_valid"]
    for k in ("cos", "l2", "tr", "total"):
        assert loss[k] == pytest.approx(o["loss"][k], rel=1e-4, abs=1e-9), k
    for name, dev_t, x0, g in (("f", st.f, s.f, o["df"]), ("K", st.K, s.K, o["dK"]), ("V", st.V, s.V, o["dV"])):
        _first_update_check(x0, dev_t.cpu().numpy().astype(np.float64), g)


def test_singleton_masks_reproduce_the_per_pixel_step(api, ctx):
    s = random_scene(11, n=3000, d=32, M=96, D=256, width=72, height=50, log_scale=-2.8, mask_drop=0.15)
    a = api.LatentStep(ctx, s, precision=api.FP32)
    b = api.LatentStep(ctx, s, precision=api.FP32, masks=pixel_masks(s))
    la = [a.step(iters=2)["total"] for _ in range(2)]
    lb = [b.step(iters=2)["total"] for _ in range(2)]
    np.testing.assert_allclose(lb, la, rtol=1e-6)
    # the two paths reduce over pixels in different orders (different row counts and splits);
    # Adam's per-coordinate normalisation turns those last-bit gradient differences into steps
    # that differ by up to lr x (relative difference) where a gradient is near zero, so the
    # parameters after four updates are compared to 1e-4 lr
    for k in ("f", "K", "V"):
        np.testing.assert_allclose(getattr(b, k).cpu().numpy(), getattr(a, k).cpu().numpy(), rtol=1e-5, atol=1e-6)


def test_step_bf16_and_stage2(api, ctx):
    s = room_scene(1, n=300_000).crop(240, 180, 160, 120)
    ms = sam_masks(s, cell=(40, 30), seed=2)
    o = om.iteration_masks(s, ms, oracle.LossConfig())
    st = api.LatentStep(ctx, s, precision=api.BF16, target_dtype=torch.bfloat16, masks=ms)
    loss = st.step(iters=1)
    for k in ("cos", "l2", "total"):
        assert loss[k] == pytest.approx(o["loss"][k], rel=5e-3, abs=1e-7), k
    # Stage II: queries fixed, the dictionary moves
    st2 = api.LatentStep(ctx, s, precision=api.FP32, masks=ms)
    f0, V0 = st2.f.clone(), st2.V.clone()
    assert np.isfinite(st2.step(iters=3, learn_f=False)["total"])
    assert torch.equal(st2.f, f0) and not torch.equal(st2.V, V0)


def test_graph_replays_match_plain_launches(api):
    s = tiny_scene(3)
    ms = sam_masks(s, cell=(16, 16), overlap=True, seed=4)
    out = []
    for graphs in (False, True):
        c = api.Context(0)
        c.graphs(graphs)
        st = api.LatentStep(c, s, precision=api.FP32, masks=ms)
        loss = [st.step(iters=2)["total"] for _ in range(4)]
        out.append(({k: getattr(st, k).cpu().numpy().copy() for k in ("f", "K", "V")}, loss))
        c.close()
    (a, la), (b, lb) = out
    np.testing.assert_allclose(lb, la, rtol=2e-5)
    for k in ("f", "K", "V"):
        assert np.linalg.norm(b[k] - a[k]) / np.linalg.norm(a[k]) <= 2e-6, k


def test_full_size_room_pooling_and_decode(api, ctx):
    """At 640x480 with 300k Gaussians and about 90 masks (the launch configuration of the
    step): the GPU's pooled queries against the oracle's pooling of the GPU's own rendered
    image, and the decode + loss + backward on the pooled rows against the oracle."""
    s = room_scene(0, n=300_000)
    ms = sam_masks(s, overlap=True, seed=0)
    proj = api.project(ctx, s.means, s.quats, s.scales, s.opacities, s.camera)
    bins = api.sort(ctx, proj, s.camera)
    Q, _, _ = api.render_fwd(ctx, proj, s.camera, bins, _dev(s.f))
    Qm = api.pool_queries(ctx, Q, ms.offsets, ms.pixels)
    Qh = Q.cpu().numpy()
    Qo = om.pool(Qh, ms.offsets, ms.pixels)
    assert _rel_rows(Qm.cpu().numpy().astype(np.float64), Qo).max() <= 1e-5
    K, V = _dev(s.K), _dev(s.V)
    parts, dQm, dK, dV = api.decode_loss_bwd(ctx, Qm, K, V, V, _dev(ms.F), _dev(ms.valid, torch.uint8),
                                             precision=api.FP32)
    cfg = oracle.LossConfig()
    Qmo = Qm.cpu().numpy().astype(np.float64)
    _, A, Fh = oracle.decode(Qmo, s.K, s.V, cfg.c(s.d))
    po, _ = oracle.loss(Fh, ms.F, ms.valid, s.V, s.V, cfg, s.d)
    gQ, gK, gV = oracle.backward(Qmo, s.K, s.V, s.V, A, Fh, ms.F, ms.valid, cfg)
    assert parts.cpu().numpy()[3] == pytest.approx(po["total"], rel=1e-5)
    for g, go in ((dQm, gQ), (dK, gK), (dV, gV)):
        g = g.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(g - go) / np.linalg.norm(go) <= 1e-3
    dQ = api.pool_queries_bwd(ctx, dQm, ms.offsets, ms.pixels, s.camera.n_pixels).cpu().numpy()
    dQo = om.pool_bwd(dQm.cpu().numpy(), ms.offsets, ms.pixels, s.camera.n_pixels)
    np.testing.assert_allclose(dQ, dQo, rtol=1e-5, atol=1e-6 * np.abs(dQo).max())


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_one_iteration_matches_oracle(api, ctx, prec):
    from workloads import room_views
    views = room_views(5, n_views=3, n=40_000, width=96, height=72, fx=78.75)
    mss = [sam_masks(v, cell=(24, 18), overlap=(k == 1), drop=0.1, seed=k) for k, v in enumerate(views)]
    p = api.FP32 if prec == "fp32" else api.BF16
    tdt = torch.float32 if prec == "fp32" else torch.bfloat16
    st = api.LatentBatchStep(ctx, views, precision=p, target_dtype=tdt, masks=mss)
    loss = st.step(iters=1)
    o = om.iteration_batch_masks(views, mss, oracle.LossConfig())
    assert loss["n_valid"] == o["loss"]["n_valid"]
    rel = 1e-4 if prec == "fp32" else 5e-3
    for k in ("cos", "l2", "total"):
        assert loss[k] == pytest.approx(o["loss"][k], rel=rel, abs=1e-9), k
    if prec == "fp32":
        _first_update_check(views[0].K, st.K.cpu().numpy().astype(np.float64), o["dK"])
        _first_update_check(views[0].V, st.V.cpu().numpy().astype(np.float64), o["dV"])
        _first_update_check(views[0].f, st.queries[0].cpu().numpy().astype(np.float64), o["df"][id(views[0].f)])


def test_latent_map_runs_algorithm_1(api, ctx):
    """Four keyframes of one room through LatentMap (B = 2, R1 = 1, R2 = 5): batch sizes grow
    with the history, the first keyframe's Stage I loss is the oracle's, and Stage II leaves the
    queries alone."""
    from workloads import room_views
    views = room_views(6, n_views=4, n=40_000, width=96, height=72, fx=78.75)
    mss = [sam_masks(v, cell=(24, 18), seed=k) for k, v in enumerate(views)]
    m = api.LatentMap(ctx, views[0], B=2)
    o = om.iteration_masks(views[0], mss[0], oracle.LossConfig())
    sizes = []
    for k, (v, ms) in enumerate(zip(views, mss)):
        r = m.add_keyframe(v.camera, masks=ms)
        sizes.append(r["batch"])
        assert np.isfinite(r["stage1"]["total"]) and np.isfinite(r["stage2"]["total"])
        if k == 0:
            assert r["stage1"]["total"] == pytest.approx(o["loss"]["total"], rel=1e-4)
    assert sizes == [1, 2, 3, 3] and len(m.history) == 4
    assert m.adam_cfg.step == 1 + 4 * (1 + 5)
    # Stage II alone: the queries stay, the dictionary moves
    m2 = api.LatentMap(ctx, views[0], B=1, R1=0, R2=3)
    f0, V0 = m2.f.clone(), m2.V.clone()
    m2.add_keyframe(views[0].camera, masks=mss[0])
    assert torch.equal(m2.f, f0) and not torch.equal(m2.V, V0)
    # the per-pixel form of the map
    m3 = api.LatentMap(ctx, views[0], B=1)
    for v in views[:2]:
        r = m3.add_keyframe(v.camera, F=v.F, mask=v.mask)
        assert np.isfinite(r["stage2"]["total"])


def test_latent_map_with_streaming_kmeans(api, ctx):
    """LatentMap with the streaming K-means first step: the atoms' weights count every valid
    mask seen, the first keyframe's update equals a direct latentam_stream_kmeans call from the
    same start, and the optimisation runs on the updated atoms."""
    from workloads import room_views
    views = room_views(8, n_views=3, n=40_000, width=96, height=72, fx=78.75)
    mss = [sam_masks(v, cell=(24, 18), seed=k) for k, v in enumerate(views)]
    m = api.LatentMap(ctx, views[0], B=1, R1=0, R2=1, kmeans=True, seed=5)
    # the same first update, directly
    rng = np.random.default_rng(5 + 1)
    rows = np.flatnonzero(mss[0].valid)
    init = rng.choice(rows, size=5, replace=False).astype(np.int32)
    V, w = _dev(views[0].V), torch.zeros(views[0].M, device="cuda")
    api.stream_kmeans(ctx, _dev(mss[0].F), V, w, init, valid=_dev(mss[0].valid, torch.uint8))
    m.R2 = 0
    m.add_keyframe(views[0].camera, masks=mss[0])
    assert torch.equal(m.V, V) and torch.equal(m.atom_weights, w)
    m.R2 = 1
    for v, ms in zip(views[1:], mss[1:]):
        r = m.add_keyframe(v.camera, masks=ms)
        assert np.isfinite(r["stage2"]["total"])
    assert float(m.atom_weights.sum()) == sum(int(ms.valid.sum()) for ms in mss)
