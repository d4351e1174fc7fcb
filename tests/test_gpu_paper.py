"""Parity of the cosine / temperature decode (the paper's W, D, tau form of Eq. dict_recon)
with the direct-form FP64 oracle (oracle/paper.py), in the FP32 and BF16 forms.

FP32: Fhat per-row relative error <= 1e-4, gradients <= 1e-3 (norm-wise), loss parts 1e-5.
BF16: the tensor-core bars of the free-key form (per-pixel cosine >= 0.999, gradients within a
relative norm error of 2e-2 and a cosine >= 0.9995, loss parts 5e-3)."""
import numpy as np
import pytest

import oracle
from oracle import paper

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


def _case(seed, n, ds, M, df, mask_drop=0.15):
    """Seeded inputs: queries ~N(0,1), W ~N(0, 1/ds), atoms ~N(0,1), half of the atoms moved
    past the trust-region radius from D0, unit targets, a random loss set."""
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(n, ds)).astype(np.float32)
    W = (rng.normal(size=(ds, df)) / np.sqrt(ds)).astype(np.float32)
    D = rng.normal(size=(M, df)).astype(np.float32)
    D0 = (D + rng.normal(size=D.shape) * 0.05 * (np.arange(M) % 2)[:, None]).astype(np.float32)
    F = rng.normal(size=(n, df))
    F = (F / np.linalg.norm(F, axis=1, keepdims=True)).astype(np.float32)
    mask = (rng.uniform(size=n) >= mask_drop).astype(np.uint8)
    return Q, W, D, D0, F, mask


SHAPES = {"ds16_M64_df128": (16, 64, 128), "ds32_M256_df512": (32, 256, 512), "ds64_M96_df384": (64, 96, 384)}
TAUS = [0.05, 0.1, 1.0]


def _rel_rows(a, b, floor):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), floor)


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("tau", TAUS)
def test_paper_fwd_fp32(api, ctx, shape, tau):
    ds, M, df = SHAPES[shape]
    Q, W, D, *_ = _case(1, 3000, ds, M, df)
    Fh, _ = api.decode_fwd_paper(ctx, _dev(Q), _dev(W), _dev(D), tau, api.FP32)
    Fo = paper.decode_paper(Q, W, D, tau)[3]
    assert _rel_rows(Fh.cpu().numpy().astype(np.float64), Fo, 1e-6).max() <= 1e-4


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("tau", TAUS)
def test_paper_loss_bwd_fp32(api, ctx, shape, tau):
    ds, M, df = SHAPES[shape]
    Q, W, D, D0, F, mask = _case(2, 2500, ds, M, df)
    cfg = oracle.LossConfig()
    Fo = paper.decode_paper(Q, W, D, tau)[3]
    po = paper.loss_paper(Fo, F, mask, D, D0, cfg)
    dQo, dWo, dDo = paper.backward_paper(Q, W, D, D0, F, mask, cfg, tau)
    parts, dQ, dW, dD = api.decode_loss_bwd_paper(ctx, _dev(Q), _dev(W), _dev(D), _dev(D0), _dev(F), tau,
                                                  _dev(mask, torch.uint8), api.LossConfig(), api.FP32)
    p = parts.cpu().numpy()
    assert p[4] == po["n_valid"]
    np.testing.assert_allclose(p[:4], [po["cos"], po["l2"], po["tr"], po["total"]], rtol=1e-5, atol=1e-9)
    for nm, g, go in (("dQ", dQ, dQo), ("dW", dW, dWo), ("dD", dD, dDo)):
        g = g.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(g - go) / np.linalg.norm(go)
        assert err <= 1e-3, (nm, err)


@pytest.mark.parametrize("shape", list(SHAPES) + ["ds32_M512_df1024"])
@pytest.mark.parametrize("tau", TAUS)
def test_paper_bf16(api, ctx, shape, tau):
    ds, M, df = SHAPES.get(shape, (32, 512, 1024))
    Q, W, D, D0, F, mask = _case(3, 2000, ds, M, df)
    cfg = oracle.LossConfig()
    Fo = paper.decode_paper(Q, W, D, tau)[3]
    Fh, _ = api.decode_fwd_paper(ctx, _dev(Q), _dev(W), _dev(D), tau, api.BF16)
    Fh = Fh.cpu().numpy().astype(np.float64)
    cos = (Fh * Fo).sum(1) / (np.linalg.norm(Fh, axis=1) * np.linalg.norm(Fo, axis=1))
    assert cos.min() >= 0.999, cos.min()
    po = paper.loss_paper(Fo, F, mask, D, D0, cfg)
    dQo, dWo, dDo = paper.backward_paper(Q, W, D, D0, F, mask, cfg, tau)
    parts, dQ, dW, dD = api.decode_loss_bwd_paper(ctx, _dev(Q), _dev(W), _dev(D), _dev(D0),
                                                  _dev(F).to(torch.bfloat16), tau, _dev(mask, torch.uint8),
                                                  api.LossConfig(), api.BF16)
    p = parts.cpu().numpy()
    np.testing.assert_allclose(p[:4], [po["cos"], po["l2"], po["tr"], po["total"]], rtol=5e-3, atol=1e-7)
    for nm, g, go in (("dQ", dQ, dQo), ("dW", dW, dWo), ("dD", dD, dDo)):
        g = g.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(g - go) / np.linalg.norm(go)
        c = float((g * go).sum() / (np.linalg.norm(g) * np.linalg.norm(go)))
        assert err <= 2e-2 and c >= 0.9995, (nm, err, c)


def test_paper_stage2_and_errors(api, ctx):
    from paper_2602_12314_gb300 import _lib as L
    Q, W, D, D0, F, mask = _case(4, 500, 32, 64, 128)
    parts, dQ, dW, dD = api.decode_loss_bwd_paper(ctx, _dev(Q), _dev(W), _dev(D), _dev(D0), _dev(F), 0.1,
                                                  _dev(mask, torch.uint8), need_dQ=False)
    assert dQ is None and np.isfinite(parts.cpu().numpy()).all()
    dWo = paper.backward_paper(Q, W, D, D0, F, mask, oracle.LossConfig(), 0.1)[1]
    assert np.linalg.norm(dW.cpu().numpy() - dWo) / np.linalg.norm(dWo) <= 1e-3
    with pytest.raises(L.LatentamError) as e:
        api.decode_fwd_paper(ctx, _dev(Q), _dev(W), _dev(D), 0.0)
    assert e.value.status == L.ERR_INVALID_ARG


def _first_update_check(x0, got, g, lr=0.01):
    x = np.asarray(x0, np.float64).copy()
    m, v = np.zeros_like(x), np.zeros_like(x)
    oracle.adam(x.reshape(-1), g.reshape(-1), m.reshape(-1), v.reshape(-1), 1, lr)
    well = (np.abs(g) > 1e-2 * np.abs(g).max()) & (np.abs(g) > 1e-5)
    np.testing.assert_allclose(got[well], x[well], rtol=0, atol=1e-4 * lr + 1e-6)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_paper_step_one_iteration_matches_oracle(api, ctx, prec):
    """latentam_step in the paper's form (tau > 0, K holding W, V the atoms D): the loss of the
    first iteration and the first Adam update of f, W and D against the oracle."""
    from workloads import tiny_scene
    s = tiny_scene(0)
    rng = np.random.default_rng(7)
    W = (rng.normal(size=(s.d, s.D)) / np.sqrt(s.d)).astype(np.float32)
    tau = 0.1
    p = api.FP32 if prec == "fp32" else api.BF16
    st = api.LatentStep(ctx, s, precision=p, target_dtype=torch.float32 if prec == "fp32" else torch.bfloat16,
                        tau=tau, W=W)
    loss = st.step(iters=1)
    cfg = oracle.LossConfig()
    proj = oracle.project_scene(s)
    Q = oracle.render_frame(proj, s.f, s.camera)[0]
    Fo = paper.decode_paper(Q, W, s.V, tau)[3]
    po = paper.loss_paper(Fo, s.F, s.mask, s.V, s.V0, cfg)
    rel = 1e-4 if prec == "fp32" else 5e-3
    assert loss["total"] == pytest.approx(po["total"], rel=rel)
    if prec == "fp32":
        dQ, dW, dD = paper.backward_paper(Q, W, s.V, s.V0, s.F, s.mask, cfg, tau)
        df = oracle.render_frame_bwd(proj, dQ, s.camera, s.n, s.d)
        _first_update_check(s.f, st.f.cpu().numpy().astype(np.float64), df)
        _first_update_check(W, st.K.cpu().numpy().astype(np.float64), dW)
        _first_update_check(s.V, st.V.cpu().numpy().astype(np.float64), dD)
    # a few more iterations stay finite and Stage II leaves f alone
    f1 = st.f.clone()
    assert np.isfinite(st.step(iters=3, learn_f=False)["total"])
    assert torch.equal(st.f, f1)


def test_paper_batch_and_map(api, ctx):
    """The batched step and LatentMap (with the streaming K-means of the atoms) in the paper's
    form: the batch's first loss against the oracle, the map's iterations finite."""
    from workloads import room_views, sam_masks
    views = room_views(4, n_views=3, n=40_000, width=96, height=72, fx=78.75)
    rng = np.random.default_rng(8)
    s0 = views[0]
    W = (rng.normal(size=(s0.d, s0.D)) / np.sqrt(s0.d)).astype(np.float32)
    st = api.LatentBatchStep(ctx, views, precision=api.FP32, tau=0.1, W=W)
    loss = st.step(iters=1)
    cfg = oracle.LossConfig()
    Q = np.concatenate([oracle.render_frame(oracle.project_scene(v), v.f, v.camera)[0] for v in views])
    F = np.concatenate([v.F for v in views])
    mask = np.concatenate([v.mask for v in views])
    po = paper.loss_paper(paper.decode_paper(Q, W, s0.V, 0.1)[3], F, mask, s0.V, s0.V0, cfg)
    assert loss["total"] == pytest.approx(po["total"], rel=1e-4)
    m = api.LatentMap(ctx, s0, B=1, kmeans=True, tau=0.1, W=W)
    for v in views:
        r = m.add_keyframe(v.camera, masks=sam_masks(v, cell=(24, 18)))
        assert np.isfinite(r["stage1"]["total"]) and np.isfinite(r["stage2"]["total"])
