"""Parity of the tensor-core decode with the FP64 oracle at pixel counts where every
persistent CTA (or cluster) of the softmax and value contractions walks several 128-row tiles.

The persistent kernels launch at most one CTA (or one cluster of CTAs sharing a row) per SM
and walk row tiles t, t + grid, t + 2 grid, ...; the second tile of a CTA uses the second TMEM
accumulator and the other box buffer, the third one wraps the barrier phases.  Small cases
reach only the first tile of each CTA, so these cases are sized for at least three tiles per
CTA / cluster on a 152-SM part (asserted from the device's SM count): the central 320 x 240
window of the room keyframe (76,800 rows, M = 256, D = 512) and random queries with the
dictionary shapes of the larger workloads (M = 512 / D = 1024 and M = 1024 / D = 768), each with
FP32 and BF16 targets.  The uneven keyframe batch (three resolutions, one M = 512, D = 768
dictionary, its rows stacked as the batched step stacks them) is compared pixel by pixel too.

Bars: per-pixel cosine(Fhat_gpu, Fhat_oracle) >= 0.999 (BF16) / 0.995 (FP8); loss parts
within 5e-3 (BF16) / 3e-2 (FP8); gradients dQ, dK, dV by relative norm (2e-2 / 0.1), tensor
cosine (0.9995 / 0.99) and per row: |g_row - o_row| / max(|o_row|, 1e-2 max|o|) <= 0.15 (BF16)
/ 0.5 (FP8).  The per-row bar follows from the BF16 rounding of A, dFhat and dS (2^-9 relative
per operand): an emulation of the BF16 form in float64 on these inputs gives at most 7e-2 on
the rows of dK (the product with the fewest terms per output), 6e-3 on dQ, 1e-4 on dV.
"""
import numpy as np
import pytest

import oracle
from workloads import keyframe_batch, room_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BARS = {
    # prec: (per-pixel cosine, loss, gradient norm, gradient cosine, per-row gradient)
    "bf16": (0.999, 5e-3, 2e-2, 0.9995, 0.15),
    "fp8": (0.995, 3e-2, 0.1, 0.99, 0.5),
}


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


def _prec(api, name):
    return {"bf16": api.BF16, "fp8": api.FP8}[name]


def _room_window():
    s = room_scene(1, n=300_000).crop(160, 120, 320, 240)
    o = oracle.project_scene(s)
    Q = oracle.render_frame(o, s.f, s.camera)[0].astype(np.float32)
    return dict(Q=Q, K=s.K, V=s.V, F=s.F, mask=s.mask)


def _random_rows(seed, n, M, D, d=32, mask_drop=0.1):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(n, d)).astype(np.float32)
    K = (rng.normal(size=(M, d)) / np.sqrt(d)).astype(np.float32)
    V = (rng.normal(size=(M, D)) / np.sqrt(d)).astype(np.float32)
    F = rng.normal(size=(n, D))
    F = (F / np.linalg.norm(F, axis=1, keepdims=True)).astype(np.float32)
    mask = (rng.uniform(size=n) >= mask_drop).astype(np.uint8)
    return dict(Q=Q, K=K, V=V, F=F, mask=mask)


CASES = {
    "room_320x240": _room_window,
    "M512_D1024": lambda: _random_rows(31, 40_000, 512, 1024),
    "M1024_D768": lambda: _random_rows(32, 24_000, 1024, 768),
}
_cache = {}


def _case(name):
    """Inputs and the oracle's decode, loss and gradients (computed once per module)."""
    if name not in _cache:
        c = CASES[name]()
        rng = np.random.default_rng(3)
        M = c["V"].shape[0]
        c["V0"] = (c["V"] + rng.normal(size=c["V"].shape) * 0.05 * (np.arange(M) % 2)[:, None]).astype(np.float32)
        cfg = oracle.LossConfig()
        d = c["Q"].shape[1]
        S, A, Fo = oracle.decode(c["Q"], c["K"], c["V"], cfg.c(d))
        c["S_max"] = S.max(1)
        c["Fhat"] = Fo
        c["parts"], _ = oracle.loss(Fo, c["F"], c["mask"], c["V"], c["V0"], cfg, d)
        c["grads"] = oracle.backward(c["Q"], c["K"], c["V"], c["V0"], A, Fo, c["F"], c["mask"], cfg)
        _cache[name] = c
    return _cache[name]


def _tiles_per_cta(n, cols):
    """Fewest row tiles a persistent CTA / cluster of ceil(cols / 256) CTAs walks."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cy = -(-cols // 256)
    tiles = -(-n // 128)
    return tiles // max(1, sms // cy)


def _cos_rows(a, b):
    return (a * b).sum(1) / np.maximum(np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1), 1e-30)


def _rel_rows(a, b, floor):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), floor)


def _check_grads(got, want, bars):
    _, _, rel_g, cos_g, row_g = bars
    for nm, g, go in zip(("dQ", "dK", "dV"), got, want):
        g = g.cpu().numpy().astype(np.float64)
        assert np.isfinite(g).all(), nm
        err = np.linalg.norm(g - go) / np.linalg.norm(go)
        cos = float((g * go).sum() / (np.linalg.norm(g) * np.linalg.norm(go)))
        rows = _rel_rows(g, go, 1e-2 * np.abs(go).max()).max()
        assert err <= rel_g and cos >= cos_g and rows <= row_g, (nm, err, cos, rows)


@pytest.mark.parametrize("prec", list(BARS))
@pytest.mark.parametrize("name", list(CASES))
def test_multitile_decode_fwd(api, ctx, name, prec):
    c = _case(name)
    n, M, D = c["Q"].shape[0], c["V"].shape[0], c["V"].shape[1]
    assert _tiles_per_cta(n, M) >= 3 and _tiles_per_cta(n, D) >= 3
    d = c["Q"].shape[1]
    Fh, stats = api.decode_fwd(ctx, _dev(c["Q"]), _dev(c["K"]), _dev(c["V"]), 1.0 / np.sqrt(d), _prec(api, prec))
    cos = _cos_rows(Fh.cpu().numpy().astype(np.float64), c["Fhat"])
    assert cos.min() >= BARS[prec][0], cos.min()
    st = stats.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(st[:, 0], c["S_max"], rtol=2e-2, atol=2e-2)


@pytest.mark.parametrize("prec", list(BARS))
@pytest.mark.parametrize("target", ["f32", "bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_multitile_decode_loss_bwd(api, ctx, name, target, prec):
    c = _case(name)
    po = c["parts"]
    F = _dev(c["F"]) if target == "f32" else _dev(c["F"]).to(torch.bfloat16)
    parts, dQ, dK, dV = api.decode_loss_bwd(ctx, _dev(c["Q"]), _dev(c["K"]), _dev(c["V"]), _dev(c["V0"]), F,
                                            _dev(c["mask"], torch.uint8), api.LossConfig(), _prec(api, prec))
    p = parts.cpu().numpy()
    assert np.isfinite(p).all()
    assert p[4] == po["n_valid"]
    np.testing.assert_allclose(p[:4], [po["cos"], po["l2"], po["tr"], po["total"]], rtol=BARS[prec][1], atol=1e-7)
    _check_grads((dQ, dK, dV), c["grads"], BARS[prec])


# ---- the uneven keyframe batch ------------------------------------------------------------

@pytest.fixture(scope="module")
def uneven():
    frames = keyframe_batch(7, sizes=((128, 96), (256, 192), (192, 144)), ns=(40_000, 120_000, 80_000))
    Qs = []
    for s in frames:
        o = oracle.project_scene(s)
        Qs.append(oracle.render_frame(o, s.f, s.camera)[0].astype(np.float32))
    Q = np.concatenate(Qs)
    F = np.concatenate([s.F for s in frames])
    mask = np.concatenate([s.mask for s in frames])
    s0 = frames[0]
    cfg = oracle.LossConfig()
    _, A, Fo = oracle.decode(Q, s0.K, s0.V, cfg.c(s0.d))
    parts, _ = oracle.loss(Fo, F, mask, s0.V, s0.V0, cfg, s0.d)
    grads = oracle.backward(Q, s0.K, s0.V, s0.V0, A, Fo, F, mask, cfg)
    return dict(frames=frames, Q=Q, F=F, mask=mask, Fhat=Fo, parts=parts, grads=grads)


@pytest.mark.parametrize("prec", list(BARS))
def test_uneven_batch_rows_per_pixel(api, ctx, uneven, prec):
    """The batched step's decode runs over the stacked rows of its keyframes (89,088 rows of
    three resolutions, M = 512, D = 768): per-pixel features, loss and gradients against the
    oracle on the same stacked rows."""
    u = uneven
    s0 = u["frames"][0]
    n = u["Q"].shape[0]
    assert _tiles_per_cta(n, s0.M) >= 3 and _tiles_per_cta(n, s0.D) >= 3
    Fh, _ = api.decode_fwd(ctx, _dev(u["Q"]), _dev(s0.K), _dev(s0.V), 1.0 / np.sqrt(s0.d), _prec(api, prec))
    cos = _cos_rows(Fh.cpu().numpy().astype(np.float64), u["Fhat"])
    assert cos.min() >= BARS[prec][0], cos.min()
    parts, dQ, dK, dV = api.decode_loss_bwd(ctx, _dev(u["Q"]), _dev(s0.K), _dev(s0.V), _dev(s0.V0),
                                            _dev(u["F"]).to(torch.bfloat16), _dev(u["mask"], torch.uint8),
                                            api.LossConfig(), _prec(api, prec))
    po = u["parts"]
    np.testing.assert_allclose(parts.cpu().numpy()[:4], [po["cos"], po["l2"], po["tr"], po["total"]],
                               rtol=BARS[prec][1], atol=1e-7)
    _check_grads((dQ, dK, dV), u["grads"], BARS[prec])


def test_uneven_batch_step_first_update(api, ctx, uneven):
    """latentam_step_batch in BF16 on the same three keyframes: the loss against the oracle's
    pooled batch iteration and the first Adam update (-lr sign(g) where |g| is far above
    Adam's epsilon) of the dictionary and of every keyframe's queries against the oracle's
    gradients, where the gradient is large enough for its sign to be determined."""
    frames = uneven["frames"]
    o = oracle.iteration_batch(frames, oracle.LossConfig())
    st = api.LatentBatchStep(ctx, frames, precision=api.BF16, target_dtype=torch.bfloat16)
    loss = st.step(iters=1, learn_f=True)
    assert loss["total"] == pytest.approx(o["loss"]["total"], rel=BARS["bf16"][1])
    lr, eps = 0.01, 1e-8
    checks = [("K", st.K, frames[0].K, o["dK"]), ("V", st.V, frames[0].V, o["dV"])]
    checks += [(f"f{k}", st.queries[k], frames[k].f, o["df"][id(frames[k].f)]) for k in range(3)]
    for nm, dev_t, x0, g in checks:
        got = dev_t.cpu().numpy().astype(np.float64)
        step = x0.astype(np.float64) - got
        # the first update is lr g / (|g| + eps): at most lr, along -sign(g) wherever the
        # gradient is large enough for its BF16 sign to be determined
        assert np.all(np.abs(step) <= lr * (1 + 1e-4) + 1e-6), nm
        well = np.abs(g) > 5e-2 * np.abs(g).max()
        assert well.sum() > 50, nm
        np.testing.assert_array_equal(np.sign(step[well]), np.sign(g[well]), err_msg=nm)
        # far above eps the step's size no longer depends on the gradient's rounding
        big = well & (np.abs(g) > 100 * eps)
        want = lr * g / (np.abs(g) + eps)
        np.testing.assert_allclose(step[big], want[big], rtol=0, atol=2e-3 * lr, err_msg=nm)
