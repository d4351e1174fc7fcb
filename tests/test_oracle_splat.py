"""Pins of the oracle's projection and query blending (Sec. III-A, Eq. alpha_blending,
Eq. render_query) against closed forms, brute force, a library rotation routine, finite
differences of the pinhole map and invariants of the blend."""
import dataclasses
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from workloads import Camera, random_scene, tiny_scene


def _axis_camera(W=48, H=40, f=50.0):
    return Camera(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=f, fy=f, cx=W / 2, cy=H / 2,
                  width=W, height=H)


def _project(means, quats, scales, opac, cam):
    return oracle.project(np.asarray(means, float), np.asarray(quats, float), np.asarray(scales, float),
                          np.asarray(opac, float), cam)


def _pinhole(cam, p):
    R = np.asarray(cam.R, float)
    pc = R @ p + np.asarray(cam.t, float)
    return np.array([cam.fx * pc[0] / pc[2] + cam.cx, cam.fy * pc[1] / pc[2] + cam.cy])


def test_projected_covariance_matches_scipy_rotation_and_numeric_jacobian():
    rng = np.random.default_rng(3)
    cam = dataclasses.replace(_axis_camera(), R=Rotation.from_euler("xyz", [0.1, -0.2, 0.3]).as_matrix(),
                              t=np.array([0.1, -0.05, 3.0]))
    for _ in range(20):
        mean = rng.uniform(-0.5, 0.5, 3)
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        s = np.exp(rng.normal(-3, 0.5, 3))
        out = _project(mean[None], q[None], s[None], [0.7], cam)
        assert out["visible"][0] == 1
        # scipy quaternions are scalar-last
        Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sigma = Rq @ np.diag(s * s) @ Rq.T
        h = 1e-6
        J = np.stack([(_pinhole(cam, mean + h * e) - _pinhole(cam, mean - h * e)) / (2 * h) for e in np.eye(3)], 1)
        cov = J @ Sigma @ J.T + 0.3 * np.eye(2)
        got = out["cov2d"][0]
        np.testing.assert_allclose([got[0], got[1], got[2]], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(out["xy"][0], _pinhole(cam, mean), rtol=1e-12)
        inv = np.linalg.inv(cov)
        np.testing.assert_allclose(out["conic"][0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-6)


def test_culling_near_plane_and_opacity():
    cam = _axis_camera()
    means = [[0, 0, 0.1], [0, 0, 0.2], [0, 0, 0.21], [0, 0, 2.0], [0, 0, -1.0]]
    q = [[1, 0, 0, 0]] * 5
    s = [[0.01] * 3] * 5
    out = _project(means, q, s, [0.5, 0.5, 0.5, 1.0 / 256, 0.5], cam)
    assert list(out["visible"]) == [0, 0, 1, 0, 0]


def test_rect_covers_every_pixel_with_alpha_at_least_threshold():
    """Brute force over every pixel: alpha >= 1/255 only inside the Gaussian's tile rect."""
    s = random_scene(5, n=300, d=4, M=4, D=8, width=70, height=45, log_scale=-2.5)
    proj = oracle.project_scene(s)
    W, H = s.camera.width, s.camera.height
    ys, xs = np.mgrid[0:H, 0:W]
    checked = 0
    for g in np.nonzero(proj["visible"])[0]:
        dx = proj["xy"][g, 0] - xs
        dy = proj["xy"][g, 1] - ys
        c = proj["conic"][g]
        a = s.opacities[g] * np.exp(-0.5 * (c[0] * dx * dx + c[2] * dy * dy) - c[1] * dx * dy)
        hit = a >= 1 / 255
        if not hit.any():
            continue
        tx, ty = xs[hit] // 16, ys[hit] // 16
        r = proj["rect"][g]
        assert (tx >= r[0]).all() and (tx < r[2]).all() and (ty >= r[1]).all() and (ty < r[3]).all()
        checked += 1
    assert checked > 50


def _iso_scene(z, s, o, f, W=48, H=40, focal=50.0, offset=(0.0, 0.0)):
    cam = _axis_camera(W, H, focal)
    means = [[offset[0], offset[1], zz] for zz in z]
    n = len(z)
    proj = _project(means, [[1, 0, 0, 0]] * n, [[ss] * 3 for ss in s], o, cam)
    return cam, proj


def test_single_isotropic_gaussian_closed_form():
    cam, proj = _iso_scene([2.5], [0.03], [0.8], None)
    f = np.array([[1.5, -2.0, 0.25]])
    Q, T, nc, amb = oracle.render_frame(proj, f, cam)
    sig2 = (cam.fx * 0.03 / 2.5) ** 2 + 0.3
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    r2 = (xs - cam.cx) ** 2 + (ys - cam.cy) ** 2
    alpha = np.minimum(0.99, 0.8 * np.exp(-r2 / (2 * sig2))).reshape(-1)
    alpha[alpha < 1 / 255] = 0.0
    np.testing.assert_allclose(Q, alpha[:, None] * f, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(T, 1 - alpha, rtol=1e-12)
    assert (nc == (alpha > 0)).all()
    assert not amb.any()


def test_two_gaussians_on_axis_and_depth_swap():
    f = np.array([[1.0, 0.0], [0.0, 1.0]])
    for z, (front, back) in [([2.0, 3.0], (0, 1)), ([3.0, 2.0], (1, 0))]:
        cam, proj = _iso_scene(z, [0.02, 0.05], [0.6, 0.9], None)
        Q, T, nc, _ = oracle.render_frame(proj, f, cam)
        ys, xs = np.mgrid[0:cam.height, 0:cam.width]
        r2 = ((xs - cam.cx) ** 2 + (ys - cam.cy) ** 2).reshape(-1)
        a = []
        for g, (zz, ss, oo) in enumerate(zip(z, [0.02, 0.05], [0.6, 0.9])):
            sig2 = (cam.fx * ss / zz) ** 2 + 0.3
            al = np.minimum(0.99, oo * np.exp(-r2 / (2 * sig2)))
            al[al < 1 / 255] = 0
            a.append(al)
        exp = np.zeros_like(Q)
        exp[:, front] = a[front]
        exp[:, back] = (1 - a[front]) * a[back]
        np.testing.assert_allclose(Q, exp, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(T, (1 - a[0]) * (1 - a[1]), rtol=1e-12)


def test_early_stop_closed_form():
    """Eight alpha = 0.8 layers: T = 0.2^k; the 6th would take T to 6.4e-5 < 1e-4, so
    exactly five contribute and T_final = 0.2^5."""
    cam = _axis_camera(16, 16, 50.0)
    n = 8
    z = 2.0 + 0.1 * np.arange(n)
    # a huge scale makes alpha ~ min(0.99, o) = o over the whole 16x16 frame
    proj = _project([[0, 0, zz] for zz in z], [[1, 0, 0, 0]] * n, [[5.0] * 3] * n, [0.8] * n, cam)
    f = np.eye(n)
    Q, T, nc, _ = oracle.render_frame(proj, f, cam)
    centre = (cam.height // 2) * cam.width + cam.width // 2
    al = 0.8 * math.exp(-0.5 * 0.0)
    assert nc[centre] == 5
    np.testing.assert_allclose(T[centre], (1 - al) ** 5, rtol=1e-9)
    exp = [al * (1 - al) ** k for k in range(5)] + [0.0] * 3
    np.testing.assert_allclose(Q[centre], exp, rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1])
def test_untiled_equals_brute_force_equals_tiled(seed):
    s = random_scene(seed, n=150, d=5, M=4, D=8, width=37, height=29, log_scale=-2.3)
    proj = oracle.project_scene(s)
    Qf, Tf, ncf, ambf = oracle.render_frame(proj, s.f, s.camera)
    W, H = s.camera.width, s.camera.height
    ys, xs = np.mgrid[0:H, 0:W]
    Qb, Tb, ncb, ambb = oracle.render_pixels(proj, s.f, xs.reshape(-1), ys.reshape(-1))
    np.testing.assert_array_equal(Qf, Qb)
    np.testing.assert_array_equal(Tf, Tb)
    np.testing.assert_array_equal(ncf, ncb)
    np.testing.assert_array_equal(ambf, ambb)
    off, ids = oracle.tile_lists(proj, s.camera)
    Qt, Tt, nct = oracle.render_tiled(proj, s.f, s.camera, off, ids)
    np.testing.assert_array_equal(Qf, Qt)
    np.testing.assert_array_equal(Tf, Tt)
    np.testing.assert_array_equal(ncf, nct)
    assert ncf.max() > 3


def test_tile_lists_sorted_by_depth_key_then_index():
    s = tiny_scene(0)
    proj = oracle.project_scene(s)
    off, ids = oracle.tile_lists(proj, s.camera)
    key = proj["depth"].astype(np.float32).astype(np.float64)
    for t in range(len(off) - 1):
        seg = ids[off[t]:off[t + 1]]
        k = list(zip(key[seg], seg))
        assert k == sorted(k)
        # membership = rect contains the tile
        tx, ty = t % ((s.camera.width + 15) // 16), t // ((s.camera.width + 15) // 16)
        r = proj["rect"]
        member = np.nonzero(proj["visible"].astype(bool) & (r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3]))[0]
        assert sorted(seg.tolist()) == member.tolist()


def test_tile_lists_break_depth_ties_by_index():
    """Many Gaussians on three depths (equal binary32 keys), rects over different tiles,
    some invisible: each tile's list is its visible members by (binary32 depth, index), the
    tie rule every renderer here shares (brute force over the synthetic projection)."""
    s = tiny_scene(0)
    tiles_x = (s.camera.width + 15) // 16
    tiles_y = (s.camera.height + 15) // 16
    rng = np.random.default_rng(7)
    N = 300
    depth = rng.choice([1.5, 2.5, 2.5 + 1e-9], size=N)  # the last two share a binary32 key
    x0 = rng.integers(0, tiles_x, size=N)
    y0 = rng.integers(0, tiles_y, size=N)
    x1 = np.minimum(tiles_x, x0 + rng.integers(1, 3, size=N))
    y1 = np.minimum(tiles_y, y0 + rng.integers(1, 3, size=N))
    proj = dict(depth=depth.astype(np.float64), visible=(rng.uniform(size=N) > 0.1).astype(np.int32),
                rect=np.ascontiguousarray(np.stack([x0, y0, x1, y1], 1).astype(np.int32)))
    off, ids = oracle.tile_lists(proj, s.camera)
    key = depth.astype(np.float32)
    assert len(np.unique(key)) == 2
    for t in range(tiles_x * tiles_y):
        tx, ty = t % tiles_x, t // tiles_x
        member = [g for g in range(N) if proj["visible"][g] and x0[g] <= tx < x1[g] and y0[g] <= ty < y1[g]]
        want = sorted(member, key=lambda g: (key[g], g))
        assert ids[off[t]:off[t + 1]].tolist() == want, t


def test_blend_weights_sum_to_one_minus_transmittance_and_linearity():
    s = tiny_scene(1)
    proj = oracle.project_scene(s)
    ones = np.ones((s.n, 1))
    Q1, T, nc, _ = oracle.render_frame(proj, ones, s.camera)
    np.testing.assert_allclose(Q1[:, 0], 1 - T, atol=1e-12)
    assert (T >= 1e-4).all() and (T <= 1).all()
    rng = np.random.default_rng(0)
    f, g = rng.normal(size=(s.n, 3)), rng.normal(size=(s.n, 3))
    Qf = oracle.render_frame(proj, f, s.camera)[0]
    Qg = oracle.render_frame(proj, g, s.camera)[0]
    Qfg = oracle.render_frame(proj, 2.5 * f - g, s.camera)[0]
    np.testing.assert_allclose(Qfg, 2.5 * Qf - Qg, atol=1e-12)


def test_transmittance_non_increasing_along_contributors():
    """T after k contributions, read off by rendering with one-hot queries of the
    front-most Gaussians, never increases."""
    s = random_scene(2, n=60, d=2, M=2, D=2, width=20, height=20, log_scale=-2.0)
    proj = oracle.project_scene(s)
    order = np.lexsort((np.arange(s.n), proj["depth"].astype(np.float32)))
    W = oracle.render_frame(proj, np.eye(s.n), s.camera)[0]  # (pixels, N) blend weights
    ones = W.sum(1)
    T = oracle.render_frame(proj, np.ones((s.n, 1)), s.camera)[1]
    np.testing.assert_allclose(ones, 1 - T, atol=1e-12)
    cum = np.cumsum(W[:, order], axis=1)
    Tk = 1 - cum
    assert (np.diff(Tk, axis=1) <= 1e-15).all()


def test_render_backward_is_transpose_of_blend_matrix():
    s = random_scene(4, n=80, d=3, M=2, D=2, width=24, height=18, log_scale=-2.2)
    proj = oracle.project_scene(s)
    Wm = oracle.render_frame(proj, np.eye(s.n), s.camera)[0]  # (pixels, N)
    rng = np.random.default_rng(1)
    dQ = rng.normal(size=(s.camera.n_pixels, 3))
    df = oracle.render_frame_bwd(proj, dQ, s.camera, s.n, 3)
    np.testing.assert_allclose(df, Wm.T @ dQ, atol=1e-12)
