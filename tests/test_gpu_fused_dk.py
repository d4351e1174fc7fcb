"""dK = c dS^T Q (the derivative of Eq. feat_loss through the softmax of Eq. dict_recon with
respect to the keys) on its two tensor-core paths, against the FP64 oracle and against each other.

With dQ requested and M <= 512, dK is the second trailing product of the dA -> dS kernel: the dS
tile staged in shared memory (never stored) times the tile's block of Q, one partial per
128-pixel tile, summed in tile order.  Without dQ (or for M > 512) dS is stored and a separate
GEMM reduces it over a pixel split.  Both read the same staged dS values and the same Q planes,
so they may differ only by FP32 summation order (bar: 1e-4 of the norm, far below any layout
or indexing mistake, which is O(1)); each must also meet its precision's oracle bars (FP32 split
form: 1e-3 by norm, 5e-3 per row; BF16: 2e-2 by norm, 0.15 per row, as the other tensor-core
tests).  Cases: a ragged pixel count (26 full tiles and a 5-row tail), M = 288 (a second CTA
per row holding 32 atoms) with d = 16, and d = 64 with M = 64 (atoms of the tile's second
128-atom group all absent).
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BARS = {"fp32": (1e-3, 5e-3), "bf16": (2e-2, 0.15)}


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


def _rows(seed, n, M, D, d):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(n, d)).astype(np.float32)
    K = (rng.normal(size=(M, d)) / np.sqrt(d)).astype(np.float32)
    V = (rng.normal(size=(M, D)) / np.sqrt(d)).astype(np.float32)
    F = rng.normal(size=(n, D))
    F = (F / np.linalg.norm(F, axis=1, keepdims=True)).astype(np.float32)
    mask = (rng.uniform(size=n) >= 0.1).astype(np.uint8)
    V0 = (V + rng.normal(size=V.shape) * 0.05 * (np.arange(M) % 2)[:, None]).astype(np.float32)
    return Q, K, V, V0, F, mask


CASES = {
    "ragged_n3333": (41, 3333, 256, 512, 32),
    "M288_d16": (42, 2000, 288, 384, 16),
    "M64_d64": (43, 1500, 64, 384, 64),
}


@pytest.mark.parametrize("prec", list(BARS))
@pytest.mark.parametrize("name", list(CASES))
def test_fused_dK_matches_oracle_and_gemm_path(api, ctx, name, prec):
    Q, K, V, V0, F, mask = _rows(*CASES[name])
    cfg = oracle.LossConfig()
    _, A, Fo = oracle.decode(Q, K, V, cfg.c(Q.shape[1]))
    _, dKo, _ = oracle.backward(Q, K, V, V0, A, Fo, F, mask, cfg)
    p = {"fp32": api.FP32, "bf16": api.BF16}[prec]
    args = (_dev(Q), _dev(K), _dev(V), _dev(V0), _dev(F), _dev(mask, torch.uint8), api.LossConfig(), p)
    _, dQ, dK_fused, _ = api.decode_loss_bwd(ctx, *args)
    _, dQ_none, dK_gemm, _ = api.decode_loss_bwd(ctx, *args, need_dQ=False)
    assert dQ is not None and dQ_none is None
    rel_g, row_g = BARS[prec]
    got = {}
    for path, g in (("fused", dK_fused), ("gemm", dK_gemm)):
        g = g.cpu().numpy().astype(np.float64)
        assert np.isfinite(g).all(), path
        err = np.linalg.norm(g - dKo) / np.linalg.norm(dKo)
        rows = (np.linalg.norm(g - dKo, axis=1) /
                np.maximum(np.linalg.norm(dKo, axis=1), 1e-2 * np.abs(dKo).max())).max()
        assert err <= rel_g and rows <= row_g, (path, err, rows)
        got[path] = g
    diff = np.linalg.norm(got["fused"] - got["gemm"]) / np.linalg.norm(got["gemm"])
    assert diff <= 1e-4, diff
