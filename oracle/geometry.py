"""Float64 oracle of the full Stage I objective and its gradients with respect to every Gaussian
attribute (Eq. full_obj: lambda_rgb L_rgb + lambda_d L_d + lambda_f L_f, with Eq. rgb_loss,
Eq. depth_loss and Eq. feat_loss), written as a differentiable PyTorch CPU program.

TEST INFRASTRUCTURE ONLY (imported by tests/ and never by the product path).

The forward restates, vectorised over all (pixel, Gaussian) pairs and without tiles, what the
C oracle computes one pixel at a time: the EWA projection (0.3 px^2 dilation, near plane,
opacity cull), the depth order (binary32 keys of the double-precision camera depth, ties by
index), alpha = min(0.99, o exp(power)) with contributions below 1/255 or with a positive
exponent skipped, front-to-back transmittance, and the stop before a contribution that would
take T below 1e-4.  The blend is applied to the queries f, the colours c (view-independent, no
spherical harmonics) and the camera depth z of each Gaussian (the rendered depth uses the same
alpha blending).  Gradients come from torch.autograd; the discrete decisions (culling, the
thresholds, the order and the stop) carry no gradient, as in the renderer.

Readings (the paper gives the losses and lambda_I1 = 0.2, lambda_I2 = 0.8, lambda_d = 0.1,
lambda_f = 5, not lambda_rgb nor the SSIM details):
  * lambda_rgb = 1;
  * L1 = mean over pixels and the three channels of |I_hat - I|;
  * L_SSIM = 1 - mean over pixels and channels of the SSIM map with an 11 x 11 Gaussian window
    (sigma 1.5), zero padding, C1 = 0.01^2, C2 = 0.03^2 (the loss of the renderer the paper
    builds on);
  * L_d = mean over the pixels with an observed depth (Z > 0) of |Z_hat - Z|;
  * L_f as in oracle.loss (the free-key decode, trust region on V).

Parity status: pinned by tests/test_oracle_geometry.py (the forward equals the C oracle's
untiled render of the stacked channels; SSIM closed forms; central finite differences of the
total with respect to means, quaternions, scales, opacities, colours, queries, keys, values).
"""
from __future__ import annotations

import math

import numpy as np
import torch

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4
DILATION = 0.3


def _t(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.float64)


def project(means, quats, scales, opac, cam):
    """Screen means (N x 2), conics (a, b, c), camera depth z (differentiable), the binary32
    sort keys and the visibility mask."""
    R = _t(cam.R).reshape(3, 3)
    t = _t(cam.t)
    # sort key: the camera depth in double with the rounding order of the renderer, to binary32
    p32 = np.asarray(means.detach().numpy(), np.float32).astype(np.float64)
    Rn = np.asarray(cam.R, np.float32).reshape(3, 3).astype(np.float64)
    zk = ((Rn[2, 0] * p32[:, 0] + Rn[2, 1] * p32[:, 1]) + Rn[2, 2] * p32[:, 2]) + float(np.float32(cam.t[2]))
    key = zk.astype(np.float32)
    cp = means @ R.T + t
    x, y, z = cp[:, 0], cp[:, 1], cp[:, 2]
    q = quats / torch.linalg.norm(quats, dim=1, keepdim=True)
    w, qx, qy, qz = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    Rq = torch.stack([
        torch.stack([1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - w * qz), 2 * (qx * qz + w * qy)], -1),
        torch.stack([2 * (qx * qy + w * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - w * qx)], -1),
        torch.stack([2 * (qx * qz - w * qy), 2 * (qy * qz + w * qx), 1 - 2 * (qx * qx + qy * qy)], -1)], -2)
    M = Rq * scales[:, None, :]  # R(q) S
    Sigma = M @ M.transpose(1, 2)
    # the camera scalars enter every implementation as binary32 values
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    zero = torch.zeros_like(z)
    J = torch.stack([torch.stack([fx / z, zero, -fx * x / (z * z)], -1),
                     torch.stack([zero, fy / z, -fy * y / (z * z)], -1)], -2)
    JW = J @ R
    S2 = JW @ Sigma @ JW.transpose(1, 2)
    ca, cb, cc = S2[:, 0, 0] + DILATION, S2[:, 0, 1], S2[:, 1, 1] + DILATION
    det = ca * cc - cb * cb
    conic = torch.stack([cc / det, -cb / det, ca / det], -1)
    uv = torch.stack([fx * x / z + cx, fy * y / z + cy], -1)
    o = opac.detach().numpy()
    vis = (zk > float(np.float32(cam.z_near))) & ~(o < ALPHA_MIN) & (det.detach().numpy() > 0)
    return uv, conic, z, key, vis


def render(uv, conic, opac, channels, key, vis, cam):
    """Front-to-back blend of `channels` (N x C) at every pixel: (H*W x C) image and T_final."""
    idx = np.flatnonzero(vis)
    order = idx[np.lexsort((idx, key[idx]))]  # by (key, index)
    o = torch.as_tensor(order)
    uv, conic, op, ch = uv[o], conic[o], opac[o], channels[o]
    W, H = cam.width, cam.height
    py, px = np.divmod(np.arange(W * H), W)
    dx = uv[None, :, 0] - _t(px)[:, None]
    dy = uv[None, :, 1] - _t(py)[:, None]
    power = -0.5 * conic[None, :, 0] * dx * dx - conic[None, :, 1] * dx * dy - 0.5 * conic[None, :, 2] * dy * dy
    raw = op[None, :] * torch.exp(power)
    alpha = torch.clamp(raw, max=ALPHA_MAX)
    take = (power.detach() <= 0) & (alpha.detach() >= ALPHA_MIN)
    alpha = torch.where(take, alpha, torch.zeros_like(alpha))
    one_minus = 1.0 - alpha
    T_after = torch.cumprod(one_minus, dim=1)
    T_before = torch.cat([torch.ones_like(T_after[:, :1]), T_after[:, :-1]], dim=1)
    stop = take & (T_after.detach() < T_MIN)
    before_stop = (torch.cumsum(stop.to(torch.int64), dim=1) - stop.to(torch.int64)) == 0
    keep = take & before_stop & ~stop
    w = torch.where(keep, alpha * T_before, torch.zeros_like(alpha))
    image = w @ ch
    return image


def gaussian_window(size: int = 11, sigma: float = 1.5) -> torch.Tensor:
    g = torch.tensor([math.exp(-((k - size // 2) ** 2) / (2 * sigma * sigma)) for k in range(size)],
                     dtype=torch.float64)
    g = g / g.sum()
    return torch.outer(g, g)


def ssim_map(a, b, C1=0.01 ** 2, C2=0.03 ** 2):
    """SSIM map of two (C, H, W) images, per channel, 11 x 11 Gaussian window, zero padding."""
    win = gaussian_window()[None, None].expand(a.shape[0], 1, 11, 11)
    conv = lambda x: torch.nn.functional.conv2d(x[None], win, padding=5, groups=a.shape[0])[0]  # noqa: E731
    mx, my = conv(a), conv(b)
    sxx = conv(a * a) - mx * mx
    syy = conv(b * b) - my * my
    sxy = conv(a * b) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def objective(params: dict, scene, image, depth, cfg, lam_rgb=1.0, lam_I1=0.2, lam_I2=0.8, lam_d=0.1):
    """The total of Eq. (full_obj) and its parts, from differentiable float64 tensors."""
    uv, conic, z, key, vis = project(params["means"], params["quats"], params["scales"], params["opacities"],
                                     scene.camera)
    d = params["f"].shape[1]
    ch = torch.cat([params["f"], params["colours"], z[:, None]], dim=1)
    img = render(uv, conic, params["opacities"], ch, key, vis, scene.camera)
    Q, C, Z = img[:, :d], img[:, d:d + 3], img[:, d + 3]
    # L_f: free-key decode and the feature loss with the trust region
    c = cfg.c(d)
    A = torch.softmax(c * Q @ params["K"].T, dim=1)
    Fh = A @ params["V"]
    F = _t(scene.F)
    m = torch.as_tensor(np.asarray(scene.mask) != 0)
    nv = max(int(m.sum()), 1)
    nF = torch.linalg.norm(F, dim=1)
    nH = torch.linalg.norm(Fh, dim=1)
    cos = (Fh * F).sum(1) / torch.clamp(nH * nF, min=1e-8)
    l_cos = ((1 - cos) * m).sum() / nv
    l_2 = (((Fh - F) ** 2).sum(1) * m).sum() / (nv * F.shape[1])
    dv = torch.linalg.norm(params["V"] - _t(scene.V0), dim=1)
    l_tr = torch.relu(dv - cfg.delta).sum()
    L_f = cfg.lambda_f * (cfg.lambda_cos * l_cos + cfg.lambda_2 * l_2 + cfg.lambda_D * l_tr)
    # L_rgb and L_d
    H, W = scene.camera.height, scene.camera.width
    I = _t(image).reshape(H * W, 3)
    l1 = (C - I).abs().mean()
    Ci = C.T.reshape(3, H, W)
    Ii = I.T.reshape(3, H, W)
    l_ssim = 1.0 - ssim_map(Ci, Ii).mean()
    L_rgb = lam_I1 * l1 + lam_I2 * l_ssim
    Zo = _t(depth)
    vd = Zo > 0
    L_d = ((Z - Zo).abs() * vd).sum() / max(int(vd.sum()), 1)
    total = lam_rgb * L_rgb + lam_d * L_d + L_f
    return total, dict(L_f=L_f, l1=l1, ssim=l_ssim, L_rgb=L_rgb, L_d=L_d, Q=Q, C=C, Z=Z)


PARAMS = ("means", "quats", "scales", "opacities", "colours", "f", "K", "V")


def gradients(scene, colours, image, depth, cfg, **lams) -> dict:
    """Total, parts and the gradient of the total with respect to every parameter group."""
    vals = dict(means=scene.means, quats=scene.quats, scales=scene.scales, opacities=scene.opacities,
                colours=colours, f=scene.f, K=scene.K, V=scene.V)
    params = {k: _t(v).clone().requires_grad_(True) for k, v in vals.items()}
    total, parts = objective(params, scene, image, depth, cfg, **lams)
    total.backward()
    out = {k: params[k].grad.numpy().copy() for k in PARAMS}
    out["total"] = float(total.detach())
    out.update({k: (float(v.detach()) if v.dim() == 0 else v.detach().numpy()) for k, v in parts.items()})
    return out
