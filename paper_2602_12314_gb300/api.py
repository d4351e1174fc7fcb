"""Python binding of the C ABI in include/latentam.h (same names, torch tensors in and out).

Argument marshalling only: tensors must live on the context's CUDA device; every step of
the computation runs in liblatentam.so's kernels.  The calls are enqueued on the current
torch CUDA stream.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math

import torch

from . import _lib as L

FP32 = L.PREC_FP32
BF16 = L.PREC_BF16
FP8 = L.PREC_FP8
FP32_FMA = L.PREC_FP32_FMA


def _lib():
    return L.load()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(None)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_f32(t, device):
    return torch.as_tensor(t, dtype=torch.float32, device=device).contiguous()


def camera_struct(cam) -> L.Camera:
    """From any object with R (3x3), t (3), fx, fy, cx, cy, width, height[, z_near]."""
    c = L.Camera()
    R = [float(x) for x in torch.as_tensor(cam.R, dtype=torch.float64).reshape(-1).tolist()]
    t = [float(x) for x in torch.as_tensor(cam.t, dtype=torch.float64).reshape(-1).tolist()]
    for k in range(9):
        c.R[k] = R[k]
    for k in range(3):
        c.t[k] = t[k]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.z_near = float(getattr(cam, "z_near", 0.2))
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def num_tiles(camera) -> int:
    c = camera if isinstance(camera, L.Camera) else camera_struct(camera)
    return int(_lib().latentam_num_tiles(ctypes.byref(c)))


@dataclasses.dataclass
class LossConfig:
    """Eq. (feat_loss) weights and lambda_f of Eq. (full_obj); defaults from Sec. IV-A.
    logit_scale <= 0 selects 1/sqrt(d)."""
    lambda_f: float = 5.0
    lambda_cos: float = 0.5
    lambda_2: float = 0.5
    lambda_D: float = 0.2
    delta: float = 0.1
    logit_scale: float = 0.0

    def struct(self) -> L.LossCfg:
        s = L.LossCfg()
        s.lambda_f, s.lambda_cos, s.lambda_2 = self.lambda_f, self.lambda_cos, self.lambda_2
        s.lambda_D, s.delta, s.logit_scale = self.lambda_D, self.delta, self.logit_scale
        return s


@dataclasses.dataclass
class AdamConfig:
    lr_f: float = 0.01
    lr_dict: float = 0.01
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    step: int = 1

    def struct(self) -> L.AdamCfg:
        s = L.AdamCfg()
        s.lr_f, s.lr_dict, s.beta1, s.beta2, s.eps, s.step = (self.lr_f, self.lr_dict, self.beta1, self.beta2,
                                                               self.eps, int(self.step))
        return s


class Context:
    """A latentam_ctx bound to one CUDA device (its workspace lives there)."""

    def __init__(self, device: int | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("latentam needs a CUDA device (GB300, sm_103a); there is no CPU fallback")
        self.device = torch.cuda.current_device() if device is None else int(device)
        lib = _lib()
        h = ctypes.c_void_p()
        L.check(lib.latentam_ctx_create(self.device, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("context destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            L.check(_lib().latentam_ctx_destroy(self._h))
            self._h = None

    def graphs(self, enable: bool = True):
        """Capture and replay the step's iterations as CUDA graphs (on by default)."""
        L.check(_lib().latentam_graphs_enable(self.handle, int(bool(enable))))

    def test_wait_timeout(self, which: int):
        """Arms a bounded device wait to give up (latentam_test_wait_timeout): 0 = the radix
        look-back of the next binning, 1 = the tensor-core kernels' wait flag."""
        L.check(_lib().latentam_test_wait_timeout(self.handle, int(which)))

    def autotune(self, enable: bool = True):
        """Time candidate tile shapes and split factors of the pixel reductions on first use of a
        shape (on by default)."""
        L.check(_lib().latentam_autotune_enable(self.handle, int(bool(enable))))

    def autotune_choices(self) -> list:
        """The autotuner's choices (latentam_autotune_query), as dicts."""
        lib = _lib()
        count = L.I32(0)
        L.check(lib.latentam_autotune_query(self.handle, 0, None, ctypes.byref(count)))
        out = []
        for i in range(count.value):
            c = L.TuneChoice()
            L.check(lib.latentam_autotune_query(self.handle, i, ctypes.byref(c), ctypes.byref(count)))
            out.append({"n": c.n, "M": c.M, "D": c.D, "reduction": c.reduction, "tile": c.tile, "split": c.split,
                        "ms": c.ms})
        return out

    def profile(self, enable: bool = True):
        """Turn the per-stage CUDA-event timers on or off."""
        L.check(_lib().latentam_profile_enable(self.handle, int(bool(enable))))

    def profile_read(self, reset: bool = True) -> dict:
        """{stage: (total ms, launch groups)} accumulated since the last reset (synchronises)."""
        ms = (ctypes.c_double * len(L.STAGES))()
        cnt = (ctypes.c_int64 * len(L.STAGES))()
        L.check(_lib().latentam_profile_read(self.handle, ms, cnt, int(bool(reset))))
        return {name: (ms[i], cnt[i]) for i, name in enumerate(L.STAGES)}

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclasses.dataclass
class Projection:
    xy: torch.Tensor             # (N, 2)
    conic_opacity: torch.Tensor  # (N, 4)
    depth: torch.Tensor          # (N,)
    rect: torch.Tensor           # (N, 4) int32
    tiles_touched: torch.Tensor  # (N,) int32

    @property
    def n(self) -> int:
        return self.depth.shape[0]

    def struct(self) -> L.Projected:
        return L.Projected(self.xy.data_ptr(), self.conic_opacity.data_ptr(), self.depth.data_ptr(),
                           self.rect.data_ptr(), self.tiles_touched.data_ptr())


@dataclasses.dataclass
class TileBins:
    pair_ids: torch.Tensor     # (capacity,) int32, first num_pairs valid
    tile_ranges: torch.Tensor  # (tiles, 2) int32
    num_pairs: int

    def struct(self) -> L.Bins:
        b = L.Bins()
        b.pair_ids = self.pair_ids.data_ptr()
        b.capacity = self.pair_ids.numel()
        b.tile_ranges = self.tile_ranges.data_ptr()
        b.num_pairs = self.num_pairs
        return b


def _gaussians_struct(means, quats, scales, opacities) -> L.Gaussians:
    g = L.Gaussians()
    g.n = means.shape[0]
    g.means, g.quats, g.scales, g.opacities = (means.data_ptr(), quats.data_ptr(), scales.data_ptr(),
                                               opacities.data_ptr())
    return g


def project(ctx: Context, means, quats, scales, opacities, camera) -> Projection:
    dev = torch.device("cuda", ctx.device)
    means, quats, scales, opacities = (_dev_f32(x, dev) for x in (means, quats, scales, opacities))
    N = means.shape[0]
    proj = Projection(torch.empty((N, 2), dtype=torch.float32, device=dev),
                      torch.empty((N, 4), dtype=torch.float32, device=dev),
                      torch.empty((N,), dtype=torch.float32, device=dev),
                      torch.empty((N, 4), dtype=torch.int32, device=dev),
                      torch.empty((N,), dtype=torch.int32, device=dev))
    g = _gaussians_struct(means, quats, scales, opacities)
    cam = camera if isinstance(camera, L.Camera) else camera_struct(camera)
    ps = proj.struct()
    L.check(_lib().latentam_project(ctx.handle, ctypes.byref(g), ctypes.byref(cam), ctypes.byref(ps), _stream()))
    return proj


def sort(ctx: Context, proj: Projection, camera, capacity: int | None = None) -> TileBins:
    """Bin and depth-sort; synchronises once to learn the pair count (retries when the
    initial buffer is too small)."""
    dev = torch.device("cuda", ctx.device)
    cam = camera if isinstance(camera, L.Camera) else camera_struct(camera)
    tiles = num_tiles(cam)
    cap = capacity if capacity is not None else max(1024, 4 * proj.n)
    ranges = torch.empty((tiles, 2), dtype=torch.int32, device=dev)
    for _ in range(2):
        bins = TileBins(torch.empty((max(cap, 1),), dtype=torch.int32, device=dev), ranges, 0)
        bs = bins.struct()
        ps = proj.struct()
        st = _lib().latentam_sort(ctx.handle, proj.n, ctypes.byref(ps), ctypes.byref(cam), ctypes.byref(bs), _stream())
        bins.num_pairs = int(bs.num_pairs)
        if st == L.ERR_CAPACITY:
            cap = bins.num_pairs
            continue
        L.check(st)
        return bins
    raise RuntimeError("pair capacity retry failed")


def render_fwd(ctx: Context, proj: Projection, camera, bins: TileBins, f: torch.Tensor):
    """Q (H*W, d), T_final (H*W,), n_contrib (H*W,) int32."""
    cam = camera if isinstance(camera, L.Camera) else camera_struct(camera)
    f = f.contiguous()
    d = f.shape[1]
    npix = cam.width * cam.height
    Q = torch.empty((npix, d), dtype=torch.float32, device=f.device)
    T = torch.empty((npix,), dtype=torch.float32, device=f.device)
    nc = torch.empty((npix,), dtype=torch.int32, device=f.device)
    ps, bs = proj.struct(), bins.struct()
    L.check(_lib().latentam_render_fwd(ctx.handle, proj.n, ctypes.byref(ps), ctypes.byref(cam), ctypes.byref(bs),
                                       _ptr(f), d, _ptr(Q), _ptr(T), _ptr(nc), _stream()))
    return Q, T, nc


def render_bwd(ctx: Context, proj: Projection, camera, bins: TileBins, n_contrib, dQ) -> torch.Tensor:
    cam = camera if isinstance(camera, L.Camera) else camera_struct(camera)
    dQ = dQ.contiguous().float()
    d = dQ.shape[1]
    df = torch.empty((proj.n, d), dtype=torch.float32, device=dQ.device)
    ps, bs = proj.struct(), bins.struct()
    L.check(_lib().latentam_render_bwd(ctx.handle, proj.n, ctypes.byref(ps), ctypes.byref(cam), ctypes.byref(bs),
                                       _ptr(n_contrib), _ptr(dQ), d, _ptr(df), _stream()))
    return df


def decode_fwd(ctx: Context, Q, K, V, logit_scale: float = 0.0, precision: int = FP32, want_stats: bool = True):
    """Fhat = softmax(c Q K^T) V and the per-row (max, sum) of the softmax."""
    Q, K, V = Q.contiguous(), K.contiguous(), V.contiguous()
    n, d = Q.shape
    M, D = V.shape
    Fh = torch.empty((n, D), dtype=torch.float32, device=Q.device)
    stats = torch.empty((n, 2), dtype=torch.float32, device=Q.device) if want_stats else None
    L.check(_lib().latentam_decode_fwd(ctx.handle, _ptr(Q), n, d, _ptr(K), _ptr(V), M, D, float(logit_scale),
                                       int(precision), _ptr(Fh), _ptr(stats), _stream()))
    return Fh, stats


def _target_dtype(F):
    if F.dtype == torch.float32:
        return L.DTYPE_F32
    if F.dtype == torch.bfloat16:
        return L.DTYPE_BF16
    raise TypeError("target features must be float32 or bfloat16")


def decode_loss_bwd(ctx: Context, Q, K, V, V0, F, mask=None, cfg: LossConfig | None = None, precision: int = FP32,
                    need_dQ: bool = True):
    """(loss_parts (5,) float64 on device, dQ, dK, dV) of lambda_f L_f, Eq. (feat_loss)."""
    cfg = cfg or LossConfig()
    Q, K, V, V0, F = (x.contiguous() for x in (Q, K, V, V0, F))
    n, d = Q.shape
    M, D = V.shape
    dev = Q.device
    parts = torch.empty((L.LOSS_PARTS,), dtype=torch.float64, device=dev)
    dQ = torch.empty((n, d), dtype=torch.float32, device=dev) if need_dQ else None
    dK = torch.empty((M, d), dtype=torch.float32, device=dev)
    dV = torch.empty((M, D), dtype=torch.float32, device=dev)
    m = mask.contiguous().to(torch.uint8) if mask is not None else None
    cs = cfg.struct()
    L.check(_lib().latentam_decode_loss_bwd(ctx.handle, _ptr(Q), n, d, _ptr(K), _ptr(V), _ptr(V0), M, D, _ptr(F),
                                            _target_dtype(F), _ptr(m), ctypes.byref(cs), int(precision), _ptr(parts),
                                            _ptr(dQ), _ptr(dK), _ptr(dV), _stream()))
    return parts, dQ, dK, dV


def stream_kmeans(ctx: Context, F, centres, weights, init_idx, valid=None, iters_local: int = 10,
                  iters_global: int = 10, want_micro: bool = False):
    """Streaming K-means update of the dictionary (Algorithm 1, Eq. stream_kmeans_init): centres
    (K x D) and weights (K) float32 device tensors are updated in place from the new embeddings
    F (n x D); init_idx holds the k_micro initial rows of the local K-means.  Returns the
    micro-clusters (centres, weights, row assignment) and the merged points' slots in the last
    global iteration when want_micro."""
    F = F.contiguous()
    n, D = F.shape
    K = centres.shape[0]
    assert centres.is_contiguous() and weights.is_contiguous() and centres.dtype == torch.float32
    idx = torch.as_tensor(init_idx, dtype=torch.int32).to(F.device).contiguous()
    k = idx.numel()
    v = valid.contiguous().to(torch.uint8) if valid is not None else None
    mC = torch.empty((k, D), dtype=torch.float32, device=F.device) if want_micro else None
    mW = torch.empty((k,), dtype=torch.float32, device=F.device) if want_micro else None
    ma = torch.empty((n,), dtype=torch.int32, device=F.device) if want_micro else None
    pa = torch.empty((K + k,), dtype=torch.int32, device=F.device) if want_micro else None
    L.check(_lib().latentam_stream_kmeans(ctx.handle, _ptr(F), n, D, _ptr(v), _ptr(idx), k, int(iters_local),
                                          int(iters_global), _ptr(centres), _ptr(weights), K, _ptr(mC), _ptr(mW),
                                          _ptr(ma), _ptr(pa), _stream()))
    return (mC, mW, ma, pa) if want_micro else None


@dataclasses.dataclass
class ImageConfig:
    """Weights of Eq. (full_obj) and Eq. (rgb_loss): lambda_rgb (no value in the paper: 1) and
    lambda_I1 = 0.2, lambda_I2 = 0.8, lambda_d = 0.1 of Sec. IV-A."""
    lambda_rgb: float = 1.0
    lambda_I1: float = 0.2
    lambda_I2: float = 0.8
    lambda_d: float = 0.1

    def struct(self) -> L.ImageCfg:
        return L.ImageCfg(self.lambda_rgb, self.lambda_I1, self.lambda_I2, self.lambda_d)


def backward_full(ctx: Context, means, quats, scales, opacities, colours, f, camera, K, V, V0, F, mask, image, depth,
                  cfg: LossConfig | None = None, icfg: ImageConfig | None = None, precision: int = FP32) -> dict:
    """Gradients of the full Stage I objective (Eq. full_obj) with respect to every Gaussian
    attribute and the dictionary, and its loss parts (latentam_backward_full)."""
    cfg, icfg = cfg or LossConfig(), icfg or ImageConfig()
    dev = torch.device("cuda", ctx.device)
    t = [_dev_f32(x, dev) for x in (means, quats, scales, opacities, colours, f, K, V, V0, image, depth)]
    means, quats, scales, opacities, colours, f, K, V, V0, image, depth = t
    F = F.contiguous() if isinstance(F, torch.Tensor) else _dev_f32(F, dev)
    m = torch.as_tensor(mask, dtype=torch.uint8).to(dev).contiguous() if mask is not None else None
    g = _gaussians_struct(means, quats, scales, opacities)
    cam = camera_struct(camera)
    out = {k: torch.empty_like(v) for k, v in (("means", means), ("quats", quats), ("scales", scales),
                                               ("opacities", opacities), ("colours", colours), ("f", f), ("K", K),
                                               ("V", V))}
    parts = torch.empty(L.FULL_LOSS_PARTS, dtype=torch.float64, device=dev)
    cs, ic = cfg.struct(), icfg.struct()
    L.check(_lib().latentam_backward_full(
        ctx.handle, ctypes.byref(g), _ptr(colours), _ptr(f), f.shape[1], ctypes.byref(cam), _ptr(K), _ptr(V), _ptr(V0),
        V.shape[0], V.shape[1], _ptr(F), _target_dtype(F), _ptr(m), _ptr(image), _ptr(depth), ctypes.byref(cs),
        ctypes.byref(ic), int(precision), _ptr(parts), _ptr(out["means"]), _ptr(out["quats"]), _ptr(out["scales"]),
        _ptr(out["opacities"]), _ptr(out["colours"]), _ptr(out["f"]), _ptr(out["K"]), _ptr(out["V"]), _stream()))
    out["parts"] = parts
    return out


class LatentStepFull:
    """Stage I of Algorithm 1 with the whole objective of Eq. (full_obj): every iteration takes
    the gradients of latentam_backward_full and one Adam update (latentam_adam) of the means,
    quaternions, scales, opacities, colours, queries, keys and values.  The Gaussians' stored
    values are optimised directly (linear scales and opacities; the renderer culls an opacity
    below 1/255 and uses the scales only through the covariance)."""

    GROUPS = ("means", "quats", "scales", "opacities", "colours", "f", "K", "V")
    LR = dict(means=1e-4, quats=1e-3, scales=1e-4, opacities=1e-3, colours=2.5e-3, f=0.01, K=0.01, V=0.01)

    def __init__(self, ctx: Context, scene, colours, image, depth, cfg: LossConfig | None = None,
                 icfg: ImageConfig | None = None, adam_cfg: AdamConfig | None = None, lr: dict | None = None):
        dev = torch.device("cuda", ctx.device)
        self.ctx = ctx
        self.cfg, self.icfg = cfg or LossConfig(), icfg or ImageConfig()
        self.adam_cfg = adam_cfg or AdamConfig()
        self.lr = dict(self.LR, **(lr or {}))
        t = lambda a: _dev_f32(a, dev)  # noqa: E731
        self.p = dict(means=t(scene.means), quats=t(scene.quats), scales=t(scene.scales),
                      opacities=t(scene.opacities), colours=t(colours), f=t(scene.f), K=t(scene.K), V=t(scene.V))
        self.m = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.V0, self.F, self.mask = t(scene.V0), t(scene.F), torch.as_tensor(scene.mask, dtype=torch.uint8).to(dev)
        self.image, self.depth, self.camera = t(image), t(depth), scene.camera

    def step(self, iters: int = 1, learn_f: bool = True, want_loss: bool = True):
        """`iters` iterations; returns the loss parts of the last one (before its update), or
        None when not want_loss.  learn_f = False (Stage II) updates only the dictionary."""
        parts = None
        groups = self.GROUPS if learn_f else ("K", "V")
        for _ in range(iters):
            p = self.p
            g = backward_full(self.ctx, p["means"], p["quats"], p["scales"], p["opacities"], p["colours"], p["f"],
                              self.camera, p["K"], p["V"], self.V0, self.F, self.mask, self.image, self.depth, self.cfg,
                              self.icfg)
            parts = g["parts"]
            adam(self.ctx, [p[k] for k in groups], [g[k] for k in groups], [self.m[k] for k in groups],
                 [self.v[k] for k in groups], [self.lr[k] for k in groups], self.adam_cfg)
            self.adam_cfg.step += 1
        if not want_loss or parts is None:
            return None
        out = parts.cpu().numpy()
        return dict(cos=out[0], l2=out[1], tr=out[2], L_f=out[3], n_valid=out[4], l1=out[5], ssim=out[6], L_d=out[7],
                    n_depth=out[8], total=out[9])


def _mask_csr(offsets, pixels, device):
    off = torch.as_tensor(offsets, dtype=torch.int32).to(device).contiguous()
    pix = torch.as_tensor(pixels, dtype=torch.int32).to(device).contiguous()
    return off, pix


def pool_queries(ctx: Context, Q, offsets, pixels):
    """Per-mask mean of the rows of Q (npix x d) over CSR mask lists (SAM-based targets,
    Sec. III-B): returns Qm (S x d)."""
    Q = Q.contiguous()
    npix, d = Q.shape
    off, pix = _mask_csr(offsets, pixels, Q.device)
    S = off.numel() - 1
    Qm = torch.empty((max(S, 0), d), dtype=torch.float32, device=Q.device)
    L.check(_lib().latentam_pool_queries(ctx.handle, _ptr(Q), npix, d, _ptr(off), _ptr(pix), pix.numel(), S,
                                         _ptr(Qm), _stream()))
    return Qm


def pool_queries_bwd(ctx: Context, dQm, offsets, pixels, npix: int):
    """Adjoint of pool_queries: dQ (npix x d) with dQ_p = sum over masks m listing p of dQm_m / |m|."""
    dQm = dQm.contiguous()
    S, d = dQm.shape
    off, pix = _mask_csr(offsets, pixels, dQm.device)
    dQ = torch.empty((npix, d), dtype=torch.float32, device=dQm.device)
    L.check(_lib().latentam_pool_queries_bwd(ctx.handle, _ptr(dQm), S, d, _ptr(off), _ptr(pix), pix.numel(),
                                             int(npix), _ptr(dQ), _stream()))
    return dQ


def decode_fwd_paper(ctx: Context, Q, W, D, tau: float, precision: int = FP32, want_stats: bool = True):
    """The paper's cosine / temperature decode (Eq. dict_recon): Fhat = softmax(cos(Q W, D) / tau) D."""
    Q, W, D = Q.contiguous(), W.contiguous(), D.contiguous()
    n, ds = Q.shape
    M, df = D.shape
    Fh = torch.empty((n, df), dtype=torch.float32, device=Q.device)
    stats = torch.empty((n, 2), dtype=torch.float32, device=Q.device) if want_stats else None
    L.check(_lib().latentam_decode_fwd_paper(ctx.handle, _ptr(Q), n, ds, _ptr(W), _ptr(D), M, df, float(tau),
                                             int(precision), _ptr(Fh), _ptr(stats), _stream()))
    return Fh, stats


def decode_loss_bwd_paper(ctx: Context, Q, W, D, D0, F, tau: float, mask=None, cfg: LossConfig | None = None,
                          precision: int = FP32, need_dQ: bool = True):
    """(loss_parts, dQ, dW, dD) of lambda_f L_f for the cosine / temperature decode, with the
    trust region on the atoms D against D0."""
    cfg = cfg or LossConfig()
    Q, W, D, D0, F = (x.contiguous() for x in (Q, W, D, D0, F))
    n, ds = Q.shape
    M, df = D.shape
    dev = Q.device
    parts = torch.empty((L.LOSS_PARTS,), dtype=torch.float64, device=dev)
    dQ = torch.empty((n, ds), dtype=torch.float32, device=dev) if need_dQ else None
    dW = torch.empty((ds, df), dtype=torch.float32, device=dev)
    dD = torch.empty((M, df), dtype=torch.float32, device=dev)
    m = mask.contiguous().to(torch.uint8) if mask is not None else None
    cs = cfg.struct()
    L.check(_lib().latentam_decode_loss_bwd_paper(ctx.handle, _ptr(Q), n, ds, _ptr(W), _ptr(D), _ptr(D0), M, df,
                                                  float(tau), _ptr(F), _target_dtype(F), _ptr(m), ctypes.byref(cs),
                                                  int(precision), _ptr(parts), _ptr(dQ), _ptr(dW), _ptr(dD),
                                                  _stream()))
    return parts, dQ, dW, dD


def decode_loss_bwd_noalloc(ctx: Context, Q, K, V, V0, F, mask=None, cfg: LossConfig | None = None,
                            out=None):
    """latentam_decode_loss_bwd_noalloc: FP32 decode + loss + backward whose scratch lives in
    the library's static device array (no device allocation inside the call).  `out`
    (optional) = preallocated (loss_parts, dQ, dK, dV) to write into."""
    cfg = cfg or LossConfig()
    Q, K, V, V0, F = (x.contiguous() for x in (Q, K, V, V0, F))
    n, d = Q.shape
    M, D = V.shape
    if out is None:
        dev = Q.device
        out = (torch.empty((L.LOSS_PARTS,), dtype=torch.float64, device=dev),
               torch.empty((n, d), dtype=torch.float32, device=dev),
               torch.empty((M, d), dtype=torch.float32, device=dev),
               torch.empty((M, D), dtype=torch.float32, device=dev))
    parts, dQ, dK, dV = out
    m = mask.contiguous().to(torch.uint8) if mask is not None else None
    cs = cfg.struct()
    L.check(_lib().latentam_decode_loss_bwd_noalloc(ctx.handle, _ptr(Q), n, d, _ptr(K), _ptr(V), _ptr(V0), M, D,
                                                    _ptr(F), _target_dtype(F), _ptr(m), ctypes.byref(cs),
                                                    _ptr(parts), _ptr(dQ), _ptr(dK), _ptr(dV), _stream()))
    return parts, dQ, dK, dV


def backward(ctx: Context, proj: Projection, camera, bins: TileBins, n_contrib, Q, K, V, V0, F, mask=None,
             cfg: LossConfig | None = None, precision: int = FP32, need_df: bool = True):
    """(loss_parts, df or None, dK, dV, dQ or None) of one keyframe."""
    cfg = cfg or LossConfig()
    cam = camera if isinstance(camera, L.Camera) else camera_struct(camera)
    Q, K, V, V0, F = (x.contiguous() for x in (Q, K, V, V0, F))
    npix, d = Q.shape
    M, D = V.shape
    dev = Q.device
    parts = torch.empty((L.LOSS_PARTS,), dtype=torch.float64, device=dev)
    dQ = torch.empty((npix, d), dtype=torch.float32, device=dev) if need_df else None
    df = torch.empty((proj.n, d), dtype=torch.float32, device=dev) if need_df else None
    dK = torch.empty((M, d), dtype=torch.float32, device=dev)
    dV = torch.empty((M, D), dtype=torch.float32, device=dev)
    m = mask.contiguous().to(torch.uint8) if mask is not None else None
    cs = cfg.struct()
    ps, bs = proj.struct(), bins.struct()
    L.check(_lib().latentam_backward(ctx.handle, proj.n, ctypes.byref(ps), ctypes.byref(cam), ctypes.byref(bs),
                                     _ptr(n_contrib), _ptr(Q), d, _ptr(K), _ptr(V), _ptr(V0), M, D, _ptr(F),
                                     _target_dtype(F), _ptr(m), ctypes.byref(cs), int(precision), _ptr(parts),
                                     _ptr(dQ), _ptr(df), _ptr(dK), _ptr(dV), _stream()))
    return parts, df, dK, dV, dQ


def adam(ctx: Context, params, grads, ms, vs, lrs, cfg: AdamConfig):
    """In-place Adam on up to 8 float32 tensors in one launch (cfg.step is NOT advanced)."""
    k = len(params)
    arr = lambda ts: (ctypes.c_void_p * k)(*[t.data_ptr() for t in ts])  # noqa: E731
    sizes = (ctypes.c_int64 * k)(*[t.numel() for t in params])
    lr = (ctypes.c_float * k)(*[float(x) for x in lrs])
    cs = cfg.struct()
    L.check(_lib().latentam_adam(ctx.handle, k, arr(params), arr(grads), arr(ms), arr(vs), sizes, lr,
                                 ctypes.byref(cs), _stream()))


class LatentStep:
    """Device-resident state of one keyframe's latent-feature optimisation (Algorithm 1,
    Stage I with learn_f = True / Stage II with learn_f = False) driven through
    latentam_step."""

    def __init__(self, ctx: Context, scene, cfg: LossConfig | None = None, adam_cfg: AdamConfig | None = None,
                 precision: int = FP32, target_dtype=torch.float32, masks=None, tau: float = 0.0, W=None):
        """`masks` (optional; offsets, pixels, per-mask targets F and flags valid, as
        workloads.MaskSet): the mask-pooled step, one decoded row and target per mask.
        tau > 0: the paper's cosine / temperature decode, with the projection W (d x D,
        required) held in K and the atoms D in V."""
        dev = torch.device("cuda", ctx.device)
        self.ctx = ctx
        self.cfg = cfg or LossConfig()
        self.adam_cfg = adam_cfg or AdamConfig()
        self.precision = int(precision)
        t = lambda a: _dev_f32(a, dev)  # noqa: E731
        self.means, self.quats, self.scales, self.opacities = (t(scene.means), t(scene.quats), t(scene.scales),
                                                               t(scene.opacities))
        self.f, self.K, self.V, self.V0 = t(scene.f), t(scene.K), t(scene.V), t(scene.V0)
        self.tau = float(tau)
        if self.tau > 0:
            if W is None:
                raise ValueError("the paper's form needs the projection W (d x D)")
            self.K = t(W)
        self.mask_offsets = self.mask_pixels = None
        if masks is None:
            self.F = t(scene.F).to(target_dtype).contiguous()
            self.mask = torch.as_tensor(scene.mask, dtype=torch.uint8, device=dev).contiguous()
        else:
            self.F = t(masks.F).to(target_dtype).contiguous()
            self.mask = torch.as_tensor(masks.valid, dtype=torch.uint8, device=dev).contiguous()
            self.mask_offsets, self.mask_pixels = _mask_csr(masks.offsets, masks.pixels, dev)
        self.moments = {k: torch.zeros_like(getattr(self, k)) for k in ("f", "K", "V")}
        self.moments.update({"v" + k: torch.zeros_like(getattr(self, k)) for k in ("f", "K", "V")})
        self.camera = camera_struct(scene.camera)
        self.d, self.M, self.D = self.f.shape[1], self.V.shape[0], self.V.shape[1]

    def frame_struct(self) -> L.Frame:
        fr = L.Frame()
        fr.gaussians = _gaussians_struct(self.means, self.quats, self.scales, self.opacities)
        fr.camera = self.camera
        fr.F = self.F.data_ptr()
        fr.F_dtype = _target_dtype(self.F)
        fr.mask = self.mask.data_ptr()
        if self.mask_offsets is not None:
            fr.mask_offsets, fr.mask_pixels = self.mask_offsets.data_ptr(), self.mask_pixels.data_ptr()
            fr.n_mask_entries = self.mask_pixels.numel()
            fr.n_masks = self.mask_offsets.numel() - 1
        return fr

    def params_struct(self) -> L.Params:
        p = L.Params()
        p.f, p.K, p.V, p.V0 = self.f.data_ptr(), self.K.data_ptr(), self.V.data_ptr(), self.V0.data_ptr()
        m = self.moments
        p.m_f, p.v_f, p.m_K, p.v_K, p.m_V, p.v_V = (m["f"].data_ptr(), m["vf"].data_ptr(), m["K"].data_ptr(),
                                                    m["vK"].data_ptr(), m["V"].data_ptr(), m["vV"].data_ptr())
        p.d, p.M, p.D = self.d, self.M, self.D
        p.tau = self.tau
        return p

    def step(self, iters: int = 1, learn_f: bool = True, want_loss: bool = True):
        """Runs `iters` fwd+bwd+Adam iterations; returns the last iteration's loss parts
        (host floats) when want_loss, else None (no synchronisation at the end)."""
        fr, pr = self.frame_struct(), self.params_struct()
        cs = self.cfg.struct()
        ac = self.adam_cfg.struct()
        out = (ctypes.c_double * L.LOSS_PARTS)() if want_loss else None
        L.check(_lib().latentam_step(self.ctx.handle, ctypes.byref(fr), ctypes.byref(pr), ctypes.byref(cs),
                                     ctypes.byref(ac), int(iters), int(bool(learn_f)), self.precision,
                                     out, _stream()))
        self.adam_cfg.step = int(ac.step)
        if out is None:
            return None
        return dict(cos=out[0], l2=out[1], tr=out[2], total=out[3], n_valid=out[4])


class LatentBatchStep:
    """Device-resident state of a batch of keyframes sharing one dictionary (the new keyframe
    plus sampled history keyframes of Algorithm 1), driven through latentam_step_batch.
    Scenes whose query arrays are the same object render one shared query tensor."""

    def __init__(self, ctx: Context, scenes, cfg: LossConfig | None = None, adam_cfg: AdamConfig | None = None,
                 precision: int = FP32, target_dtype=torch.float32, masks=None, tau: float = 0.0, W=None):
        """`masks` (optional): one mask set per scene (workloads.MaskSet layout), the
        mask-pooled batch.  tau > 0 and W: the paper's decode, as in LatentStep."""
        if not 1 <= len(scenes) <= L.MAX_BATCH:
            raise ValueError(f"a batch holds 1..{L.MAX_BATCH} keyframes")
        dev = torch.device("cuda", ctx.device)
        self.ctx = ctx
        self.cfg = cfg or LossConfig()
        self.adam_cfg = adam_cfg or AdamConfig()
        self.precision = int(precision)
        t = lambda a: _dev_f32(a, dev)  # noqa: E731
        s0 = scenes[0]
        self.K, self.V, self.V0 = t(s0.K), t(s0.V), t(s0.V0)
        self.tau = float(tau)
        if self.tau > 0:
            if W is None:
                raise ValueError("the paper's form needs the projection W (d x D)")
            self.K = t(W)
        self.mK, self.vK = torch.zeros_like(self.K), torch.zeros_like(self.K)
        self.mV, self.vV = torch.zeros_like(self.V), torch.zeros_like(self.V)
        self.d, self.M, self.D = s0.f.shape[1], self.V.shape[0], self.V.shape[1]
        geo, qs = {}, {}
        self.frames = []
        for sc in scenes:
            gk = id(sc.means)
            if gk not in geo:
                geo[gk] = tuple(t(getattr(sc, a)) for a in ("means", "quats", "scales", "opacities"))
            qk = id(sc.f)
            if qk not in qs:
                f = t(sc.f)
                qs[qk] = (f, torch.zeros_like(f), torch.zeros_like(f))
            self.frames.append((geo[gk], qs[qk], camera_struct(sc.camera)))
        self.queries = [q[0] for q in qs.values()]
        self.csr = None
        if masks is None:
            self.F = torch.cat([t(sc.F) for sc in scenes]).to(target_dtype).contiguous()
            self.mask = torch.cat([torch.as_tensor(sc.mask, dtype=torch.uint8) for sc in scenes]).to(dev).contiguous()
        else:
            if len(masks) != len(scenes):
                raise ValueError("one mask set per scene")
            self.F = torch.cat([t(m.F) for m in masks]).to(target_dtype).contiguous()
            self.mask = torch.cat([torch.as_tensor(m.valid, dtype=torch.uint8) for m in masks]).to(dev).contiguous()
            self.csr = [_mask_csr(m.offsets, m.pixels, dev) for m in masks]

    def step(self, iters: int = 1, learn_f: bool = True, want_loss: bool = True):
        fr = (L.BatchFrame * len(self.frames))()
        for k, (g, q, cam) in enumerate(self.frames):
            fr[k].gaussians = _gaussians_struct(*g)
            fr[k].camera = cam
            fr[k].f, fr[k].m_f, fr[k].v_f = q[0].data_ptr(), q[1].data_ptr(), q[2].data_ptr()
            if self.csr is not None:
                off, pix = self.csr[k]
                fr[k].mask_offsets, fr[k].mask_pixels = off.data_ptr(), pix.data_ptr()
                fr[k].n_mask_entries, fr[k].n_masks = pix.numel(), off.numel() - 1
        dic = L.Dictionary(self.K.data_ptr(), self.V.data_ptr(), self.V0.data_ptr(), self.mK.data_ptr(),
                           self.vK.data_ptr(), self.mV.data_ptr(), self.vV.data_ptr(), self.d, self.M, self.D, self.tau)
        cs = self.cfg.struct()
        ac = self.adam_cfg.struct()
        out = (ctypes.c_double * L.LOSS_PARTS)() if want_loss else None
        L.check(_lib().latentam_step_batch(self.ctx.handle, fr, len(self.frames), _ptr(self.F), _target_dtype(self.F),
                                           _ptr(self.mask), ctypes.byref(dic), ctypes.byref(cs), ctypes.byref(ac),
                                           int(iters), int(bool(learn_f)), self.precision, out, _stream()))
        self.adam_cfg.step = int(ac.step)
        if out is None:
            return None
        return dict(cos=out[0], l2=out[1], tr=out[2], total=out[3], n_valid=out[4])


@dataclasses.dataclass
class Keyframe:
    """One keyframe of a LatentMap on the device: its camera, its targets (per pixel, or per
    mask with the CSR mask lists) and its loss-set flags."""
    camera: L.Camera
    F: torch.Tensor
    mask: torch.Tensor
    csr: tuple | None = None  # (offsets, pixels) int32 device tensors when mask-pooled
    valid_rows: object = None  # host indices of the rows in the loss set (K-means starts)

    @property
    def rows(self) -> int:
        return self.F.shape[0]


class LatentMap:
    """The optimisation loop of Algorithm 1 over a stream of keyframes of one map (Sec. III-C).

    The map's Gaussians and queries f and the dictionary (K, V) with their Adam moments stay on
    the device.  add_keyframe(camera, targets) runs, for the new keyframe:
      0. with kmeans: the streaming K-means update of the atoms V from the keyframe's targets
         (latentam_stream_kmeans, k_micro micro-clusters started at rows drawn by the map's
         seeded generator; the slots' weights live in `atom_weights`);
      1. the trust-region centre V0 <- V (the dictionary at the start of the keyframe);
      2. the training batch: the new keyframe plus B keyframes sampled from the history;
      3. Stage I: R1 iterations updating f, K and V (the Gaussians' other attributes are fixed);
      4. Stage II: R2 iterations updating K and V with f fixed;
      5. the new keyframe joins the history.
    Defaults R1 = 1, R2 = 5 (Sec. III-C).  Every iteration goes through latentam_step_batch.
    With a voxel_map (a VoxelMap holding the global Gaussian map, Sec. III-E), each keyframe
    first synchronises the map around its camera centre with the active radius, and the map's
    local Gaussians, queries and moments are optimised in place (the next synchronisation
    writes them back); `scene` then supplies only the dictionary."""

    def __init__(self, ctx: Context, scene, cfg: LossConfig | None = None, adam_cfg: AdamConfig | None = None,
                 precision: int = FP32, target_dtype=torch.float32, B: int = 2, R1: int = 1, R2: int = 5,
                 seed: int = 0, kmeans: bool = False, k_micro: int = 5, kmeans_iters: int = 10,
                 voxel_map=None, radius: float = 5.0, tau: float = 0.0, W=None):
        import numpy as np

        from .history import KeyframeHistory

        dev = torch.device("cuda", ctx.device)
        self.ctx, self.dev = ctx, dev
        self.cfg = cfg or LossConfig()
        self.adam_cfg = adam_cfg or AdamConfig()
        self.precision, self.target_dtype = int(precision), target_dtype
        self.B, self.R1, self.R2 = int(B), int(R1), int(R2)
        t = lambda a: _dev_f32(a, dev)  # noqa: E731
        self.voxel_map, self.radius = voxel_map, float(radius)
        if voxel_map is None:
            self.geometry = tuple(t(getattr(scene, a)) for a in ("means", "quats", "scales", "opacities"))
            self.f = t(scene.f)
            self.m_f, self.v_f = torch.zeros_like(self.f), torch.zeros_like(self.f)
        else:
            self._use_local(voxel_map.local())
        self.K, self.V = t(scene.K), t(scene.V)
        self.tau = float(tau)
        if self.tau > 0:  # the paper's decode: K holds the projection W, V the atoms D
            if W is None:
                raise ValueError("the paper's form needs the projection W (d x D)")
            self.K = t(W)
        self.V0 = self.V.clone()
        self.mK, self.vK = torch.zeros_like(self.K), torch.zeros_like(self.K)
        self.mV, self.vV = torch.zeros_like(self.V), torch.zeros_like(self.V)
        self.d, self.M, self.D = scene.f.shape[1], self.V.shape[0], self.V.shape[1]
        self.history = KeyframeHistory(seed)
        self.kmeans, self.k_micro, self.kmeans_iters = bool(kmeans), int(k_micro), int(kmeans_iters)
        self.atom_weights = torch.zeros(self.M, dtype=torch.float32, device=dev)  # every slot empty
        self._rng = np.random.default_rng(seed + 1)

    def keyframe(self, camera, F, mask=None, masks=None) -> Keyframe:
        """Device copy of a keyframe: per-pixel targets F (H*W x D) with loss-set mask, or a
        mask set (offsets, pixels, per-mask targets F and flags valid)."""
        import numpy as np

        dev = self.dev
        if masks is not None:
            return Keyframe(camera_struct(camera), _dev_f32(masks.F, dev).to(self.target_dtype).contiguous(),
                            torch.as_tensor(masks.valid, dtype=torch.uint8).to(dev).contiguous(),
                            _mask_csr(masks.offsets, masks.pixels, dev), np.flatnonzero(np.asarray(masks.valid)))
        n = camera.width * camera.height
        m = torch.ones(n, dtype=torch.uint8) if mask is None else torch.as_tensor(mask, dtype=torch.uint8)
        return Keyframe(camera_struct(camera), _dev_f32(F, dev).to(self.target_dtype).contiguous(),
                        m.to(dev).contiguous(), None, np.flatnonzero(m.numpy()))

    def _use_local(self, loc: dict):
        self.geometry = (loc["means"], loc["quats"], loc["scales"], loc["opacities"])
        self.f, self.m_f, self.v_f = loc["f"], loc["m_f"], loc["v_f"]

    def _sync(self, camera):
        R = torch.as_tensor(camera.R, dtype=torch.float64)
        t = torch.as_tensor(camera.t, dtype=torch.float64)
        centre = (-R.T @ t).tolist()  # the camera centre in world coordinates
        self._use_local(self.voxel_map.sync(centre, self.radius))

    def _update_atoms(self, kf: Keyframe):
        rows = kf.valid_rows
        if rows is None or len(rows) == 0:
            return
        k = min(self.k_micro, len(rows))
        init = self._rng.choice(rows, size=k, replace=False).astype("int32")
        F = kf.F if kf.F.dtype == torch.float32 else kf.F.float()
        stream_kmeans(self.ctx, F, self.V, self.atom_weights, init, valid=kf.mask, iters_local=self.kmeans_iters,
                      iters_global=self.kmeans_iters)

    def _run(self, batch, iters: int, learn_f: bool):
        if iters <= 0:
            return None
        pooled = batch[0].csr is not None
        if any((k.csr is not None) != pooled for k in batch):
            raise ValueError("keyframes of one map are either all mask-pooled or all per-pixel")
        fr = (L.BatchFrame * len(batch))()
        for i, kf in enumerate(batch):
            fr[i].gaussians = _gaussians_struct(*self.geometry)
            fr[i].camera = kf.camera
            fr[i].f, fr[i].m_f, fr[i].v_f = self.f.data_ptr(), self.m_f.data_ptr(), self.v_f.data_ptr()
            if pooled:
                off, pix = kf.csr
                fr[i].mask_offsets, fr[i].mask_pixels = off.data_ptr(), pix.data_ptr()
                fr[i].n_mask_entries, fr[i].n_masks = pix.numel(), off.numel() - 1
        F = torch.cat([k.F for k in batch]).contiguous()
        mask = torch.cat([k.mask for k in batch]).contiguous()
        dic = L.Dictionary(self.K.data_ptr(), self.V.data_ptr(), self.V0.data_ptr(), self.mK.data_ptr(),
                           self.vK.data_ptr(), self.mV.data_ptr(), self.vV.data_ptr(), self.d, self.M, self.D, self.tau)
        cs, ac = self.cfg.struct(), self.adam_cfg.struct()
        out = (ctypes.c_double * L.LOSS_PARTS)()
        L.check(_lib().latentam_step_batch(self.ctx.handle, fr, len(batch), _ptr(F), _target_dtype(F), _ptr(mask),
                                           ctypes.byref(dic), ctypes.byref(cs), ctypes.byref(ac), int(iters),
                                           int(bool(learn_f)), self.precision, out, _stream()))
        self.adam_cfg.step = int(ac.step)
        return dict(cos=out[0], l2=out[1], tr=out[2], total=out[3], n_valid=out[4])

    def add_keyframe(self, camera, F=None, mask=None, masks=None) -> dict:
        """Algorithm 1's optimisation of one new keyframe; returns the loss of the last Stage I
        and Stage II iterations and the batch size."""
        kf = self.keyframe(camera, F, mask, masks)
        if self.voxel_map is not None:
            self._sync(camera)
        if self.kmeans:
            self._update_atoms(kf)
        self.V0.copy_(self.V)
        batch = self.history.batch(kf, self.B)
        l1 = self._run(batch, self.R1, True)
        l2 = self._run(batch, self.R2, False)
        self.history.add(kf)
        return dict(stage1=l1, stage2=l2, batch=len(batch))


class _DeviceArray:
    """A view of map-owned device memory for torch.as_tensor (no copy)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2}


def _device_view(ptr, shape, typestr, dev):
    if ptr is None or any(s == 0 for s in shape):
        dt = torch.int32 if typestr == "<i4" else torch.float32
        return torch.empty(shape, dtype=dt, device=dev)
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device=dev)


def _host_view(ptr, shape, typestr):
    """A view of pinned host memory owned by the library (no copy)."""
    import numpy as np

    count = 1
    for s_ in shape:
        count *= s_
    if ptr is None or count == 0:
        return torch.empty(shape, dtype=torch.float32)
    ct = ctypes.c_float if typestr == "<f4" else ctypes.c_int32
    arr = np.ctypeslib.as_array((ct * count).from_address(int(ptr))).reshape(shape)
    return torch.from_numpy(arr)


class VoxelMap:
    """The voxel-hashed global Gaussian map and the active local map (Sec. III-E), held on the
    device by latentam_map.  The tensors that local() and global_store() return are views of
    the map's memory, valid until the next call that changes the map."""

    def __init__(self, ctx: Context, d: int, table_log2: int = 24, voxel_size: float = 0.01, capacity: int = 1 << 20,
                 host_store: bool = False):
        """host_store: the global store's rows in pinned host memory (the slot table and the
        local map stay on the device); global_store() then returns host tensors."""
        self.ctx, self.d = ctx, int(d)
        self.dev = torch.device("cuda", ctx.device)
        self.host_store = bool(host_store)
        h = ctypes.c_void_p()
        L.check(_lib().latentam_map_create(ctx.handle, self.d, int(table_log2), float(voxel_size), int(capacity),
                                           int(self.host_store), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            _lib().latentam_map_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _gaussians(self, means, quats, scales, opacities, f):
        t = [_dev_f32(x, self.dev) for x in (means, quats, scales, opacities, f)]
        return t, _gaussians_struct(*t[:4])

    def insert(self, means, quats, scales, opacities, f):
        """Insert-if-free in input order; returns (each row's new index or -1, count inserted)."""
        t, g = self._gaussians(means, quats, scales, opacities, f)
        out = torch.empty(g.n, dtype=torch.int32, device=self.dev)
        n = ctypes.c_int64(0)
        L.check(_lib().latentam_map_insert(self.ctx.handle, self.handle, ctypes.byref(g), _ptr(t[4]), _ptr(out),
                                           ctypes.byref(n), _stream()))
        return out, int(n.value)

    def add_local(self, means, quats, scales, opacities, f):
        t, g = self._gaussians(means, quats, scales, opacities, f)
        L.check(_lib().latentam_map_add_local(self.ctx.handle, self.handle, ctypes.byref(g), _ptr(t[4]), _stream()))
        torch.cuda.current_stream().synchronize()

    def _local_dict(self, v: L.MapLocal) -> dict:
        n, d = int(v.count), self.d
        out = {k: _device_view(getattr(v, k), (n, w), "<f4", self.dev)
               for k, w in (("means", 3), ("quats", 4), ("scales", 3), ("f", d), ("m_f", d), ("v_f", d))}
        out["opacities"] = _device_view(v.opacities, (n,), "<f4", self.dev)
        out["gidx"] = _device_view(v.gidx, (n,), "<i4", self.dev)
        return out

    def sync(self, centre, radius: float) -> dict:
        """Local -> Global then Global -> Local around `centre`; returns the new local map."""
        c = (ctypes.c_float * 3)(*[float(x) for x in centre])
        v = L.MapLocal()
        L.check(_lib().latentam_map_sync(self.ctx.handle, self.handle, c, float(radius), ctypes.byref(v), _stream()))
        return self._local_dict(v)

    def local(self) -> dict:
        v = L.MapLocal()
        L.check(_lib().latentam_map_local_view(self.handle, ctypes.byref(v)))
        return self._local_dict(v)

    def global_store(self) -> dict:
        v = L.MapGlobal()
        L.check(_lib().latentam_map_global_view(self.handle, ctypes.byref(v)))
        torch.cuda.current_stream().synchronize()
        n, d = int(v.count), self.d
        view = _host_view if self.host_store else (lambda p, shape, ts: _device_view(p, shape, ts, self.dev))
        out = {k: view(getattr(v, k), (n, w), "<f4") for k, w in (("means", 3), ("quats", 4), ("scales", 3), ("f", d))}
        out["opacities"] = view(v.opacities, (n,), "<f4")
        out["table"] = _device_view(v.table, (int(v.table_size),), "<i4", self.dev)
        return out


def default_logit_scale(d: int) -> float:
    return 1.0 / math.sqrt(d)
