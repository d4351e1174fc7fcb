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
