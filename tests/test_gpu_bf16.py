"""Parity of the BF16 tensor-core decode (tcgen05, FP32 accumulation) with the FP64 oracle.

Tolerances: decoded features per-pixel cosine >= 0.999 against the oracle (the decode's
stated bar for BF16 operands).  Loss and gradients: BF16 rounds each operand to 8
significant bits (relative 2^-9); products summed in FP32 keep that order of error, and the
backward chains three such contractions, so gradients are held to a relative norm error of
2e-2 and a tensor cosine >= 0.9995, the loss parts to a relative 5e-3.
"""
import numpy as np
import pytest

import oracle
from workloads import random_scene, room_scene, tiny_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COS_F = 0.999
REL_G = 2e-2
COS_G = 0.9995
REL_LOSS = 5e-3


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


def _case(name):
    if name == "tiny":
        return tiny_scene(0)
    if name == "ragged":
        return random_scene(11, n=3000, d=32, M=96, D=256, width=72, height=50, log_scale=-2.8, mask_drop=0.15)
    if name == "d64":
        return random_scene(12, n=1500, d=64, M=64, D=384, width=40, height=33, log_scale=-2.6)
    if name == "d16_M512":
        return random_scene(13, n=2000, d=16, M=512, D=512, width=48, height=40, log_scale=-2.6, mask_drop=0.1)
    if name == "room_crop":
        return room_scene(1, n=300_000).crop(272, 208, 96, 64)
    # the dictionary shapes of the larger workloads: rows of S and Fhat spread over clusters
    if name == "M512_D1024":
        return random_scene(14, n=3000, d=32, M=512, D=1024, width=64, height=48, log_scale=-2.7, mask_drop=0.1)
    if name == "M1024_D768":
        return random_scene(15, n=3000, d=32, M=1024, D=768, width=56, height=40, log_scale=-2.7)
    if name == "M288_D384":  # the last CTA of each cluster holds a partial slice
        return random_scene(16, n=2000, d=16, M=288, D=384, width=50, height=37, log_scale=-2.6, mask_drop=0.2)
    raise KeyError(name)


CASES = ["tiny", "ragged", "d64", "d16_M512", "room_crop", "M512_D1024", "M1024_D768", "M288_D384"]


def _oracle_Q(s):
    o = oracle.project_scene(s)
    return oracle.render_frame(o, s.f, s.camera)[0].astype(np.float32)


def _cos_rows(a, b):
    return (a * b).sum(1) / np.maximum(np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1), 1e-30)


@pytest.mark.parametrize("name", CASES)
def test_bf16_decode_fwd_cosine(api, ctx, name):
    s = _case(name)
    Q = _oracle_Q(s)
    c = 1.0 / np.sqrt(s.d)
    Fh, stats = api.decode_fwd(ctx, _dev(Q), _dev(s.K), _dev(s.V), c, api.BF16)
    S, _, Fo = oracle.decode(Q, s.K, s.V, c)
    cos = _cos_rows(Fh.cpu().numpy().astype(np.float64), Fo)
    assert cos.min() >= COS_F, cos.min()
    st = stats.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(st[:, 0], S.max(1), rtol=2e-2, atol=2e-2)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("target", ["f32", "bf16"])
def test_bf16_decode_loss_bwd(api, ctx, name, target):
    s = _case(name)
    Q = _oracle_Q(s)
    rng = np.random.default_rng(3)
    V0 = (s.V + (rng.normal(size=s.V.shape) * 0.05 * (np.arange(s.M) % 2)[:, None])).astype(np.float32)
    cfg = oracle.LossConfig()
    _, A, Fo = oracle.decode(Q, s.K, s.V, cfg.c(s.d))
    po, _ = oracle.loss(Fo, s.F, s.mask, s.V, V0, cfg, s.d)
    dQo, dKo, dVo = oracle.backward(Q, s.K, s.V, V0, A, Fo, s.F, s.mask, cfg)
    F = _dev(s.F) if target == "f32" else _dev(s.F).to(torch.bfloat16)
    parts, dQ, dK, dV = api.decode_loss_bwd(ctx, _dev(Q), _dev(s.K), _dev(s.V), _dev(V0), F,
                                            _dev(s.mask, torch.uint8), api.LossConfig(), api.BF16)
    p = parts.cpu().numpy()
    assert np.isfinite(p).all()
    assert p[4] == po["n_valid"]
    np.testing.assert_allclose(p[:4], [po["cos"], po["l2"], po["tr"], po["total"]], rtol=REL_LOSS, atol=1e-7)
    for nm, g, go in (("dQ", dQ, dQo), ("dK", dK, dKo), ("dV", dV, dVo)):
        g = g.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(g - go) / np.linalg.norm(go)
        cos = float((g * go).sum() / (np.linalg.norm(g) * np.linalg.norm(go)))
        assert err <= REL_G and cos >= COS_G, (nm, err, cos)


def test_bf16_step_matches_fp32_step(api, ctx):
    s = _case("ragged")
    l32 = api.LatentStep(ctx, s, precision=api.FP32).step(iters=1, learn_f=True)
    st = api.LatentStep(ctx, s, precision=api.BF16, target_dtype=torch.bfloat16)
    l16 = st.step(iters=1, learn_f=True)
    assert l16["total"] == pytest.approx(l32["total"], rel=REL_LOSS)
    l16b = st.step(iters=2, learn_f=True)
    assert np.isfinite(l16b["total"])


def test_bf16_rejects_oversized_rows(api, ctx):
    from paper_2602_12314_gb300 import _lib as L
    Q = torch.zeros((10, 32), device="cuda")
    with pytest.raises(L.LatentamError) as e:
        api.decode_fwd(ctx, Q, torch.zeros((64, 32), device="cuda"), torch.zeros((64, 1152), device="cuda"),
                       precision=api.BF16)
    assert e.value.status == L.ERR_UNSUPPORTED_SHAPE
