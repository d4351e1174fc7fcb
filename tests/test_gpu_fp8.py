"""Parity of the FP8 form (the value contraction Fhat = A V on E4M3 tcgen05 operands, the rest
as in the BF16 form) with the FP64 oracle.

Bars: decoded features per-pixel cosine >= 0.995 (the FP8 bar of the decode).  E4M3 keeps 3
mantissa bits (rounding error up to 2^-4 relative, about 3.6% RMS per element); the attention
rows and the values each carry it into Fhat, and the backward inherits it through dFhat =
a_p Fhat + b_p F, so gradients are held to a relative norm error of 0.1 and a tensor cosine of
0.99, loss parts to 3e-2 relative."""
import numpy as np
import pytest

import oracle
from workloads import random_scene, room_scene, tiny_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COS_F = 0.995
REL_G = 0.1
COS_G = 0.99
REL_LOSS = 3e-2


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
    if name == "room_crop":
        return room_scene(1, n=300_000).crop(272, 208, 96, 64)
    if name == "M512_D1024":
        return random_scene(14, n=3000, d=32, M=512, D=1024, width=64, height=48, log_scale=-2.7, mask_drop=0.1)
    if name == "M1024_D768":
        return random_scene(15, n=3000, d=32, M=1024, D=768, width=56, height=40, log_scale=-2.7)
    raise KeyError(name)


CASES = ["tiny", "ragged", "room_crop", "M512_D1024", "M1024_D768"]


def _oracle_Q(s):
    o = oracle.project_scene(s)
    return oracle.render_frame(o, s.f, s.camera)[0].astype(np.float32)


@pytest.mark.parametrize("name", CASES)
def test_fp8_decode_fwd_cosine(api, ctx, name):
    s = _case(name)
    Q = _oracle_Q(s)
    c = 1.0 / np.sqrt(s.d)
    Fh, stats = api.decode_fwd(ctx, _dev(Q), _dev(s.K), _dev(s.V), c, api.FP8)
    S, _, Fo = oracle.decode(Q, s.K, s.V, c)
    Fh = Fh.cpu().numpy().astype(np.float64)
    cos = (Fh * Fo).sum(1) / np.maximum(np.linalg.norm(Fh, axis=1) * np.linalg.norm(Fo, axis=1), 1e-30)
    assert cos.min() >= COS_F, cos.min()
    np.testing.assert_allclose(stats.cpu().numpy()[:, 0], S.max(1), rtol=2e-2, atol=2e-2)


@pytest.mark.parametrize("name", CASES)
def test_fp8_decode_loss_bwd(api, ctx, name):
    s = _case(name)
    Q = _oracle_Q(s)
    rng = np.random.default_rng(3)
    V0 = (s.V + (rng.normal(size=s.V.shape) * 0.05 * (np.arange(s.M) % 2)[:, None])).astype(np.float32)
    cfg = oracle.LossConfig()
    _, A, Fo = oracle.decode(Q, s.K, s.V, cfg.c(s.d))
    po, _ = oracle.loss(Fo, s.F, s.mask, s.V, V0, cfg, s.d)
    dQo, dKo, dVo = oracle.backward(Q, s.K, s.V, V0, A, Fo, s.F, s.mask, cfg)
    parts, dQ, dK, dV = api.decode_loss_bwd(ctx, _dev(Q), _dev(s.K), _dev(s.V), _dev(V0),
                                            _dev(s.F).to(torch.bfloat16), _dev(s.mask, torch.uint8),
                                            api.LossConfig(), api.FP8)
    p = parts.cpu().numpy()
    assert np.isfinite(p).all() and p[4] == po["n_valid"]
    np.testing.assert_allclose(p[:4], [po["cos"], po["l2"], po["tr"], po["total"]], rtol=REL_LOSS, atol=1e-6)
    for nm, g, go in (("dQ", dQ, dQo), ("dK", dK, dKo), ("dV", dV, dVo)):
        g = g.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(g - go) / np.linalg.norm(go)
        cs = float((g * go).sum() / (np.linalg.norm(g) * np.linalg.norm(go)))
        assert err <= REL_G and cs >= COS_G, (nm, err, cs)


def test_fp8_step_and_paper_form(api, ctx):
    s = _case("ragged")
    st = api.LatentStep(ctx, s, precision=api.FP8, target_dtype=torch.bfloat16)
    l0 = st.step(iters=1)
    l1 = st.step(iters=3)
    assert np.isfinite(l0["total"]) and np.isfinite(l1["total"])
    from oracle import paper
    rng = np.random.default_rng(9)
    Q = rng.normal(size=(2000, 32)).astype(np.float32)
    W = (rng.normal(size=(32, 512)) / np.sqrt(32)).astype(np.float32)
    D = rng.normal(size=(256, 512)).astype(np.float32)
    Fh, _ = api.decode_fwd_paper(ctx, _dev(Q), _dev(W), _dev(D), 0.1, api.FP8)
    Fo = paper.decode_paper(Q, W, D, 0.1)[3]
    Fh = Fh.cpu().numpy().astype(np.float64)
    cos = (Fh * Fo).sum(1) / (np.linalg.norm(Fh, axis=1) * np.linalg.norm(Fo, axis=1))
    assert cos.min() >= COS_F, cos.min()
