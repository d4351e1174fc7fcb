"""Parity of the full Stage I backward (latentam_backward_full: geometry, colour and depth with
Eq. full_obj) with the float64 autograd oracle of oracle/geometry.py.

Tolerances (FP32 form): loss parts within a relative 1e-4 (the SSIM mean and the sums over
pixels in FP64), every gradient tensor within a relative norm error of 1e-3 (the bar of the
other gradients; the opacity, mean and conic gradients add the suffix term of the blend, a
difference of two float32 sums), Gaussians that touch no pixel get exactly zero."""
import numpy as np
import pytest

import oracle
from oracle import geometry as geo
from workloads import random_scene, room_scene

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


def _inputs(s, seed):
    rng = np.random.default_rng(seed)
    n, npix = s.n, s.camera.n_pixels
    colours = rng.uniform(0, 1, size=(n, 3)).astype(np.float32)
    image = rng.uniform(0, 1, size=(npix, 3)).astype(np.float32)
    depth = (rng.uniform(2.0, 5.0, size=npix) * (rng.uniform(size=npix) > 0.2)).astype(np.float32)
    return colours, image, depth


def _touching(s):
    """Gaussians whose tile rect is not empty (every pixel they reach lies inside it)."""
    p = oracle.project_scene(s)
    r = p["rect"]
    return np.flatnonzero((p["visible"] != 0) & (r[:, 2] > r[:, 0]) & (r[:, 3] > r[:, 1]))


def _compare(api, ctx, s, seed, tol=1e-3):
    colours, image, depth = _inputs(s, seed)
    cfg = oracle.LossConfig()
    got = api.backward_full(ctx, s.means, s.quats, s.scales, s.opacities, colours, s.f, s.camera, s.K, s.V, s.V0,
                            s.F, s.mask, image, depth)
    keep = _touching(s)
    sub = s.__class__(**{**s.__dict__, "means": s.means[keep], "quats": s.quats[keep], "scales": s.scales[keep],
                         "opacities": s.opacities[keep], "f": s.f[keep]})
    o = geo.gradients(sub, colours[keep], image, depth, cfg)
    parts = got["parts"].cpu().numpy()
    want = [o["L_f"], o["l1"], o["ssim"], o["L_d"], o["total"]]
    np.testing.assert_allclose([parts[3], parts[5], parts[6], parts[7], parts[9]], want, rtol=1e-4)
    for k in geo.PARAMS:
        g = got[k].cpu().numpy().astype(np.float64)
        go = o[k]
        if k not in ("K", "V"):
            rest = np.ones(s.n, bool)
            rest[keep] = False
            assert np.all(g[rest] == 0.0), k
            g = g[keep]
        err = np.linalg.norm(g - go) / max(np.linalg.norm(go), 1e-30)
        assert err <= tol, (k, err)
    return got, o


def test_full_backward_random_scene(api, ctx):
    s = random_scene(31, n=400, d=16, M=32, D=128, width=40, height=30, log_scale=-2.4, mask_drop=0.15)
    _compare(api, ctx, s, 1)


def test_full_backward_d32_scene(api, ctx):
    s = random_scene(32, n=300, d=32, M=64, D=128, width=33, height=27, log_scale=-2.3)
    _compare(api, ctx, s, 2)


def test_full_backward_room_crop(api, ctx):
    """A 48 x 32 window of the room keyframe (its Gaussians that reach the window)."""
    s = room_scene(2, n=300_000).crop(296, 224, 48, 32)
    _compare(api, ctx, s, 3)


def test_full_step_first_update_and_descent(api, ctx):
    """LatentStepFull: the first Adam update of every group is -lr sign(g) of the oracle's
    gradient wherever that gradient is well above rounding, untouched Gaussians do not move, and
    twenty iterations lower the total of Eq. (full_obj)."""
    s = random_scene(33, n=300, d=16, M=32, D=128, width=40, height=30, log_scale=-2.4, mask_drop=0.1)
    colours, image, depth = _inputs(s, 4)
    st = api.LatentStepFull(ctx, s, colours, image, depth)
    first = st.step(1)
    keep = _touching(s)
    sub = s.__class__(**{**s.__dict__, "means": s.means[keep], "quats": s.quats[keep], "scales": s.scales[keep],
                         "opacities": s.opacities[keep], "f": s.f[keep]})
    o = geo.gradients(sub, colours[keep], image, depth, oracle.LossConfig())
    assert first["total"] == pytest.approx(o["total"], rel=1e-4)
    init = dict(means=s.means, quats=s.quats, scales=s.scales, opacities=s.opacities, colours=colours, f=s.f, K=s.K,
                V=s.V)
    for k in st.GROUPS:
        x0 = np.asarray(init[k], np.float64)
        got = st.p[k].cpu().numpy().astype(np.float64)
        g = o[k]
        if k not in ("K", "V"):
            rest = np.ones(s.n, bool)
            rest[keep] = False
            assert np.array_equal(got[rest], x0[rest]), k
            got, x0 = got[keep], x0[keep]
        lr = st.lr[k]
        # the first step is -lr sign(g) only where |g| is far above Adam's epsilon (1e-8)
        well = (np.abs(g) > 1e-2 * np.abs(g).max()) & (np.abs(g) > 1e-5)
        np.testing.assert_allclose(got[well], (x0 - lr * np.sign(g))[well], rtol=0, atol=1e-3 * lr + 1e-6, err_msg=k)
    last = st.step(19)
    assert last["total"] < first["total"] - 1e-2  # random targets: a slow but steady descent
