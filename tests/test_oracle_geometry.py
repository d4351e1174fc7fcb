"""Pins of the full-objective oracle (oracle/geometry.py): its vectorised forward equals the C
oracle's untiled render of the stacked channels [f | colour | depth]; SSIM's closed forms; the
gradients of the total with respect to every parameter group against central finite
differences of the forward."""
import numpy as np
import pytest

import oracle
from oracle import geometry as geo
from workloads import random_scene

torch = pytest.importorskip("torch")


def _case(seed=0, n=60, d=4, M=6, D=12, w=24, h=18):
    s = random_scene(seed, n=n, d=d, M=M, D=D, width=w, height=h, log_scale=-2.2, mask_drop=0.2)
    rng = np.random.default_rng(seed + 100)
    colours = rng.uniform(0, 1, size=(n, 3))
    image = rng.uniform(0, 1, size=(h * w, 3))
    depth = rng.uniform(2.0, 4.0, size=h * w) * (rng.uniform(size=h * w) > 0.2)
    return s, colours, image, depth


def test_forward_equals_c_oracle_render_of_stacked_channels():
    s, colours, image, depth = _case(1)
    t = lambda x: torch.as_tensor(np.asarray(x, np.float64))  # noqa: E731
    uv, conic, z, key, vis = geo.project(t(s.means), t(s.quats), t(s.scales), t(s.opacities), s.camera)
    ch = np.concatenate([s.f, colours, z.detach().numpy()[:, None]], axis=1)
    img = geo.render(uv, conic, t(s.opacities), t(ch), key, vis, s.camera).detach().numpy()
    proj = oracle.project_scene(s)
    ref, _, _, amb = oracle.render_frame(proj, ch, s.camera)
    ok = ~amb
    np.testing.assert_allclose(img[ok], ref[ok], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(uv.detach().numpy()[vis], proj["xy"][vis], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(conic.detach().numpy()[vis], proj["conic"][vis], rtol=1e-9, atol=1e-12)


def test_feature_loss_part_equals_c_oracle_loss():
    s, colours, image, depth = _case(5)
    cfg = oracle.LossConfig()
    g = geo.gradients(s, colours, image, depth, cfg)
    _, _, Fh = oracle.decode(g["Q"], s.K, s.V, cfg.c(s.d))
    parts, _ = oracle.loss(Fh, s.F, s.mask, s.V, s.V0, cfg, s.d)
    assert g["L_f"] == pytest.approx(parts["total"], rel=1e-12)
    assert g["total"] == pytest.approx(g["L_rgb"] + 0.1 * g["L_d"] + g["L_f"], rel=1e-14)


def test_ssim_closed_forms():
    rng = np.random.default_rng(2)
    a = torch.as_tensor(rng.uniform(size=(3, 20, 24)))
    np.testing.assert_allclose(geo.ssim_map(a, a).numpy(), 1.0, rtol=0, atol=1e-12)
    # constant images: in the interior (window fully inside) sigma = 0 and
    # SSIM = (2 a b + C1) / (a^2 + b^2 + C1)
    x, y = 0.3, 0.7
    A = torch.full((1, 20, 24), x, dtype=torch.float64)
    B = torch.full((1, 20, 24), y, dtype=torch.float64)
    m = geo.ssim_map(A, B).numpy()[0, 5:-5, 5:-5]
    np.testing.assert_allclose(m, (2 * x * y + 1e-4) / (x * x + y * y + 1e-4), rtol=1e-12)
    # the window sums to one and is symmetric
    w = geo.gaussian_window().numpy()
    assert abs(w.sum() - 1) < 1e-14 and np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])


def test_gradients_match_central_differences():
    s, colours, image, depth = _case(3)
    cfg = oracle.LossConfig()
    g = geo.gradients(s, colours, image, depth, cfg)
    vals = dict(means=s.means, quats=s.quats, scales=s.scales, opacities=s.opacities, colours=colours, f=s.f,
                K=s.K, V=s.V)
    base = {k: np.array(v, np.float64) for k, v in vals.items()}

    def total(p):
        params = {k: torch.as_tensor(v) for k, v in p.items()}
        return float(geo.objective(params, s, image, depth, cfg)[0])

    rng = np.random.default_rng(4)
    # Gaussians that contribute (their query gradient is non-zero)
    live = np.flatnonzero(np.abs(g["f"]).sum(1) > 0)
    assert len(live) >= 10
    for name in geo.PARAMS:
        X = base[name]
        for _ in range(5):
            if name in ("K", "V"):
                ix = tuple(int(rng.integers(0, k)) for k in X.shape)
            else:
                i = int(rng.choice(live))
                ix = (i,) if X.ndim == 1 else (i, int(rng.integers(0, X.shape[1])))
            h = 1e-6 * max(1.0, abs(X[ix]))
            p, m = dict(base), dict(base)
            p[name], m[name] = X.copy(), X.copy()
            p[name][ix] += h
            m[name][ix] -= h
            num = (total(p) - total(m)) / (2 * h)
            assert num == pytest.approx(g[name][ix], rel=1e-4, abs=1e-8), (name, ix)
