"""The CUDA-graph form of latentam_step: replayed iterations give the same parameters as plain
launches (the only difference is the Adam bias correction evaluated on the device from the
step counter, a few ulp), for both precision forms and for several iterations per call."""
import numpy as np
import pytest

from workloads import random_scene, tiny_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2602_12314_gb300 import api as _api
    return _api


def _run(api, scene, graphs, prec, calls, iters):
    ctx = api.Context(0)
    ctx.graphs(graphs)
    tdt = torch.float32 if prec == api.FP32 else torch.bfloat16
    st = api.LatentStep(ctx, scene, precision=prec, target_dtype=tdt)
    losses = [st.step(iters=iters, learn_f=True)["total"] for _ in range(calls)]
    out = {k: getattr(st, k).cpu().numpy().copy() for k in ("f", "K", "V")}
    out["step"] = st.adam_cfg.step
    out["loss"] = losses
    ctx.close()
    return out


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("iters", [1, 3])
def test_graph_replays_match_plain_launches(api, prec, iters):
    s = random_scene(21, n=3000, d=32, M=96, D=256, width=72, height=50, log_scale=-2.8, mask_drop=0.15)
    p = api.FP32 if prec == "fp32" else api.BF16
    calls = 5  # the configuration is captured on its second or third use and replayed after
    a = _run(api, s, False, p, calls, iters)
    b = _run(api, s, True, p, calls, iters)
    assert a["step"] == b["step"] == 1 + calls * iters
    # The replays differ from plain launches only by the few-ulp bias-correction rounding; in
    # the BF16 form that can flip the rounding of an operand to 8 significant bits, which a
    # few iterations carry into single entries (relative 2^-9 per flip), so its bar is wider.
    tol = 2e-5 if prec == "fp32" else 5e-4
    for k in ("f", "K", "V"):
        err = np.linalg.norm(b[k] - a[k]) / np.linalg.norm(a[k])
        assert err <= tol / 10, (k, err)
        np.testing.assert_allclose(b[k], a[k], rtol=tol, atol=tol * np.abs(a[k]).max(), err_msg=k)
    np.testing.assert_allclose(b["loss"], a["loss"], rtol=tol)


def test_graphs_follow_new_buffers(api):
    """A second keyframe (new buffers, other sizes) in the same context is captured anew."""
    ctx = api.Context(0)
    s1 = tiny_scene(0)
    s2 = random_scene(22, n=2000, d=16, M=64, D=128, width=40, height=33, log_scale=-2.6)
    for s in (s1, s2, s1):
        st = api.LatentStep(ctx, s)
        for _ in range(4):
            loss = st.step(1)
        assert np.isfinite(loss["total"])
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_graph_replays_match_plain_launches(api, prec):
    from workloads import room_views
    views = room_views(5, n_views=3, n=40_000, width=96, height=72, fx=78.75)
    p = api.FP32 if prec == "fp32" else api.BF16
    tdt = torch.float32 if prec == "fp32" else torch.bfloat16
    out = []
    for graphs in (False, True):
        ctx = api.Context(0)
        ctx.graphs(graphs)
        st = api.LatentBatchStep(ctx, views, precision=p, target_dtype=tdt)
        loss = [st.step(iters=2, learn_f=True)["total"] for _ in range(4)]
        out.append(({k: getattr(st, k).cpu().numpy().copy() for k in ("K", "V")},
                    st.queries[0].cpu().numpy().copy(), loss, st.adam_cfg.step))
        ctx.close()
    (a, fa, la, sa), (b, fb, lb, sb) = out
    assert sa == sb == 9
    tol = 2e-5 if prec == "fp32" else 5e-4
    for k in ("K", "V"):
        assert np.linalg.norm(b[k] - a[k]) / np.linalg.norm(a[k]) <= tol / 10, k
    assert np.linalg.norm(fb - fa) / np.linalg.norm(fa) <= tol / 10
    np.testing.assert_allclose(lb, la, rtol=tol)


def test_autotuned_splits_change_only_summation_order(api):
    from workloads import room_scene
    s = room_scene(4, n=60_000, width=160, height=120, fx=131.25)
    out = []
    for tune in (False, True):
        ctx = api.Context(0)
        ctx.autotune(tune)
        Q = torch.randn((s.camera.n_pixels, s.d), device="cuda", generator=torch.Generator("cuda").manual_seed(0))
        K, V = (torch.as_tensor(x, device="cuda") for x in (s.K, s.V))
        F = torch.as_tensor(s.F, device="cuda").to(torch.bfloat16)
        mask = torch.as_tensor(s.mask, device="cuda")
        res = [api.decode_loss_bwd(ctx, Q, K, V, V, F, mask, precision=api.BF16) for _ in range(2)]
        out.append([t.cpu().numpy() for t in res[-1]])
        choices = ctx.autotune_choices()
        if tune:  # one choice per reduction over pixels: dV (tile shape and split); dK (M <= 512)
            # comes from per-tile partials of the dA -> dS kernel, with no split to choose
            assert sorted(c["reduction"] for c in choices) == [5]
            for c in choices:
                assert (c["n"], c["M"], c["D"]) == (s.camera.n_pixels, s.M, s.D)
                assert c["tile"] in ((0, 1) if c["reduction"] == 5 else (0,))
                assert c["split"] >= 1 and c["ms"] > 0
        else:
            assert choices == []
        ctx.close()
    for a, b in zip(out[0], out[1]):
        np.testing.assert_allclose(b, a, rtol=1e-4, atol=1e-6 * np.abs(a).max())
