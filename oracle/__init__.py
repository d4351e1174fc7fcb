"""FP64 CPU oracle of the LatentAM latent-feature optimisation step (arxiv 2602.12314).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg; never by the product path.  The arithmetic lives in
``latentam_oracle.c`` (plain C, double precision); this module only builds it, marshals
numpy arrays in and out, and chains the steps in the order of Algorithm 1's
optimisation stage: render (Eq. render_query) -> decode (Eq. dict_recon) -> loss
(Eq. feat_loss, Eq. full_obj) -> gradients -> Adam.

Parity status: every function here is pinned by tests/test_oracle_*.py against closed
forms, brute force, invariants, library routines or central finite differences.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "latentam_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liblatentam_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction) into oracle/_build/."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "latentam_oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("z_near", ctypes.c_double), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class _LossCfg(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("lambda_f", "lambda_cos", "lambda_2", "lambda_D", "delta", "logit_scale")]


@dataclasses.dataclass
class LossConfig:
    """Weights of Eq. (feat_loss) and lambda_f of Eq. (full_obj); the values of
    Sec. IV-A are the defaults.  logit_scale c: None -> 1/sqrt(d)."""
    lambda_f: float = 5.0
    lambda_cos: float = 0.5
    lambda_2: float = 0.5
    lambda_D: float = 0.2
    delta: float = 0.1
    logit_scale: float | None = None

    def c(self, d: int) -> float:
        return float(self.logit_scale) if self.logit_scale is not None else 1.0 / np.sqrt(d)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64, I32 = ctypes.c_int64, ctypes.c_int32
            lib.orc_project.argtypes = [I64, P, P, P, P, P, P, P, P, P, P, P, P, P]
            lib.orc_project.restype = None
            lib.orc_render_frame.argtypes = [I64, I32, P, P, P, P, P, P, P, P, P, P, P, P]
            lib.orc_render_frame.restype = ctypes.c_int
            lib.orc_render_frame_bwd.argtypes = [I64, I32, P, P, P, P, P, P, P, P, P]
            lib.orc_render_frame_bwd.restype = ctypes.c_int
            lib.orc_render_pixels.argtypes = [I64, I32, P, P, P, P, P, P, I64, P, P, P, P, P, P]
            lib.orc_render_pixels.restype = None
            lib.orc_tile_lists.argtypes = [I64, P, P, P, P, I64, P, P, P]
            lib.orc_tile_lists.restype = ctypes.c_int
            lib.orc_render_tiled.argtypes = [I32, P, P, P, P, P, P, P, P, P, P]
            lib.orc_render_tiled.restype = None
            lib.orc_decode.argtypes = [I64, I32, I32, I32, P, P, P, ctypes.c_double, P, P, P]
            lib.orc_decode.restype = None
            lib.orc_loss.argtypes = [I64, I32, I32, P, P, P, P, P, P, P, P]
            lib.orc_loss.restype = None
            lib.orc_backward.argtypes = [I64, I32, I32, I32, P, P, P, P, P, P, P, P, P, P, P, P]
            lib.orc_backward.restype = None
            lib.orc_adam.argtypes = [I64, P, P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double]
            lib.orc_adam.restype = None
            _lib = lib
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def camera_struct(cam) -> _Camera:
    c = _Camera()
    R = np.asarray(cam.R, np.float64).reshape(-1)
    t = np.asarray(cam.t, np.float64).reshape(-1)
    for k in range(9):
        c.R[k] = float(R[k])
    for k in range(3):
        c.t[k] = float(t[k])
    # camera scalars enter every implementation as binary32 values
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    c.fx, c.fy, c.cx, c.cy = f32(cam.fx), f32(cam.fy), f32(cam.cx), f32(cam.cy)
    c.z_near = f32(cam.z_near)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def _cfg_struct(cfg: LossConfig, d: int) -> _LossCfg:
    s = _LossCfg()
    s.lambda_f, s.lambda_cos, s.lambda_2 = cfg.lambda_f, cfg.lambda_cos, cfg.lambda_2
    s.lambda_D, s.delta, s.logit_scale = cfg.lambda_D, cfg.delta, cfg.c(d)
    return s


# --------------------------------------------------------------------------------------
# Splatting
# --------------------------------------------------------------------------------------

def project(means, quats, scales, opacities, cam) -> dict:
    """Per-Gaussian projection: xy, cov2d (a, b, c of Sigma'), conic, depth, extent,
    tile rect (x0, y0, x1, y1, half-open), visible, rect_ambiguous."""
    lib = _load()
    means, quats, scales, opac = _d(means), _d(quats), _d(scales), _d(opacities)
    N = means.shape[0]
    out = dict(xy=np.zeros((N, 2)), cov2d=np.zeros((N, 3)), conic=np.zeros((N, 3)), depth=np.zeros(N),
               extent=np.zeros((N, 2)), rect=np.zeros((N, 4), np.int32), visible=np.zeros(N, np.int32),
               rect_ambiguous=np.zeros(N, np.int32))
    c = camera_struct(cam)
    lib.orc_project(N, _p(means), _p(quats), _p(scales), _p(opac), ctypes.byref(c),
                    _p(out["xy"]), _p(out["cov2d"]), _p(out["conic"]), _p(out["depth"]), _p(out["extent"]),
                    _p(out["rect"]), _p(out["visible"]), _p(out["rect_ambiguous"]))
    out["opacities"] = opac
    return out


def project_scene(scene) -> dict:
    return project(scene.means, scene.quats, scene.scales, scene.opacities, scene.camera)


def render_frame(proj: dict, f, cam):
    """Untiled Eq. (render_query) over the whole frame: Q (H*W, d), T_final, n_contrib, ambiguous."""
    lib = _load()
    f = _d(f)
    N, d = f.shape
    n = cam.width * cam.height
    Q, T = np.zeros((n, d)), np.zeros(n)
    nc, amb = np.zeros(n, np.int32), np.zeros(n, np.uint8)
    c = camera_struct(cam)
    rc = lib.orc_render_frame(N, d, _p(proj["xy"]), _p(proj["conic"]), _p(proj["opacities"]), _p(proj["depth"]),
                              _p(proj["visible"]), _p(proj["cov2d"]), _p(f), ctypes.byref(c),
                              _p(Q), _p(T), _p(nc), _p(amb))
    if rc:
        raise MemoryError("oracle render_frame: allocation failed")
    return Q, T, nc, amb.astype(bool)


def render_frame_bwd(proj: dict, dQ, cam, N: int, d: int) -> np.ndarray:
    """df_i = sum_p w_ip dQ_p over the untiled per-pixel lists."""
    lib = _load()
    dQ = _d(dQ)
    df = np.zeros((N, d))
    c = camera_struct(cam)
    rc = lib.orc_render_frame_bwd(N, d, _p(proj["xy"]), _p(proj["conic"]), _p(proj["opacities"]),
                                  _p(proj["depth"]), _p(proj["visible"]), _p(proj["cov2d"]), ctypes.byref(c),
                                  _p(dQ), _p(df))
    if rc:
        raise MemoryError("oracle render_frame_bwd: allocation failed")
    return df


def render_pixels(proj: dict, f, px, py):
    """Brute-force blend of the listed pixels against all Gaussians."""
    lib = _load()
    f = _d(f)
    N, d = f.shape
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    k = px.shape[0]
    Q, T = np.zeros((k, d)), np.zeros(k)
    nc, amb = np.zeros(k, np.int32), np.zeros(k, np.uint8)
    lib.orc_render_pixels(N, d, _p(proj["xy"]), _p(proj["conic"]), _p(proj["opacities"]), _p(proj["depth"]),
                          _p(proj["visible"]), _p(f), k, _p(px), _p(py), _p(Q), _p(T), _p(nc), _p(amb))
    return Q, T, nc, amb.astype(bool)


def tile_lists(proj: dict, cam):
    """Per-16x16-tile Gaussian lists sorted by (depth, index): (offsets[T+1], ids[P])."""
    lib = _load()
    N = proj["depth"].shape[0]
    c = camera_struct(cam)
    P = ctypes.c_int64(0)
    lib.orc_tile_lists(N, _p(proj["depth"]), _p(proj["visible"]), _p(proj["rect"]), ctypes.byref(c), 0,
                       ctypes.byref(P), None, None)
    nt = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    off = np.zeros(nt + 1, np.int64)
    ids = np.zeros(max(P.value, 1), np.int32)
    rc = lib.orc_tile_lists(N, _p(proj["depth"]), _p(proj["visible"]), _p(proj["rect"]), ctypes.byref(c),
                            P.value, ctypes.byref(P), _p(off), _p(ids))
    if rc:
        raise MemoryError("oracle tile_lists: allocation failed")
    return off, ids[:P.value]


def render_tiled(proj: dict, f, cam, offsets, ids):
    lib = _load()
    f = _d(f)
    d = f.shape[1]
    n = cam.width * cam.height
    Q, T, nc = np.zeros((n, d)), np.zeros(n), np.zeros(n, np.int32)
    c = camera_struct(cam)
    offsets = np.ascontiguousarray(offsets, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    lib.orc_render_tiled(d, _p(proj["xy"]), _p(proj["conic"]), _p(proj["opacities"]), _p(f), ctypes.byref(c),
                         _p(offsets), _p(ids), _p(Q), _p(T), _p(nc))
    return Q, T, nc


# --------------------------------------------------------------------------------------
# Decode, loss, gradients, optimiser
# --------------------------------------------------------------------------------------

def decode(Q, K, V, c: float):
    """Eq. (dict_recon) with free keys: returns S, A, Fhat."""
    lib = _load()
    Q, K, V = _d(Q), _d(K), _d(V)
    n, d = Q.shape
    M, D = V.shape
    S, A, Fh = np.zeros((n, M)), np.zeros((n, M)), np.zeros((n, D))
    lib.orc_decode(n, d, M, D, _p(Q), _p(K), _p(V), float(c), _p(S), _p(A), _p(Fh))
    return S, A, Fh


def loss(Fhat, F, mask, V, V0, cfg: LossConfig, d: int):
    """lambda_f * L_f; returns (dict of parts, per-pixel cos)."""
    lib = _load()
    Fhat, F, V, V0 = _d(Fhat), _d(F), _d(V), _d(V0)
    mask = np.ascontiguousarray(mask, np.uint8)
    n, D = Fhat.shape
    M = V.shape[0]
    parts = np.zeros(5)
    cos_p = np.zeros(n)
    cs = _cfg_struct(cfg, d)
    lib.orc_loss(n, M, D, _p(Fhat), _p(F), _p(mask), _p(V), _p(V0), ctypes.byref(cs), _p(parts), _p(cos_p))
    return dict(cos=parts[0], l2=parts[1], tr=parts[2], total=parts[3], n_valid=int(parts[4])), cos_p


def backward(Q, K, V, V0, A, Fhat, F, mask, cfg: LossConfig):
    """Gradients of loss(decode(Q, K, V)) with respect to Q, K, V."""
    lib = _load()
    Q, K, V, V0, A, Fhat, F = map(_d, (Q, K, V, V0, A, Fhat, F))
    mask = np.ascontiguousarray(mask, np.uint8)
    n, d = Q.shape
    M, D = V.shape
    dQ, dK, dV = np.zeros((n, d)), np.zeros((M, d)), np.zeros((M, D))
    cs = _cfg_struct(cfg, d)
    lib.orc_backward(n, d, M, D, _p(Q), _p(K), _p(V), _p(V0), _p(A), _p(Fhat), _p(F), _p(mask), ctypes.byref(cs),
                     _p(dQ), _p(dK), _p(dV))
    return dQ, dK, dV


def adam(param, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays."""
    lib = _load()
    for a in (param, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    grad = _d(grad)
    lib.orc_adam(param.size, _p(param), _p(grad), _p(m), _p(v), int(step), float(lr), float(beta1), float(beta2),
                 float(eps))


def iteration(scene, cfg: LossConfig | None = None, f=None, K=None, V=None, proj=None, with_df=True) -> dict:
    """One forward + backward of the step on a full frame (no optimiser update):
    render -> decode -> loss -> dQ, dK, dV -> df."""
    cfg = cfg or LossConfig()
    f = scene.f if f is None else f
    K = scene.K if K is None else K
    V = scene.V if V is None else V
    proj = proj if proj is not None else project_scene(scene)
    Q, T, nc, amb = render_frame(proj, f, scene.camera)
    S, A, Fh = decode(Q, K, V, cfg.c(Q.shape[1]))
    parts, cos_p = loss(Fh, scene.F, scene.mask, V, scene.V0, cfg, Q.shape[1])
    dQ, dK, dV = backward(Q, K, V, scene.V0, A, Fh, scene.F, scene.mask, cfg)
    out = dict(proj=proj, Q=Q, T=T, n_contrib=nc, ambiguous=amb, S=S, A=A, Fhat=Fh, loss=parts, cos_p=cos_p,
               dQ=dQ, dK=dK, dV=dV)
    if with_df:
        out["df"] = render_frame_bwd(proj, dQ, scene.camera, np.asarray(f).shape[0], Q.shape[1])
    return out


def iteration_batch(scenes, cfg: LossConfig | None = None) -> dict:
    """One forward + backward over a batch of keyframes sharing the dictionary: each frame
    rendered untiled, the loss pooled over the loss-set pixels of all frames (targets and
    masks concatenated in frame order), one trust-region term; df summed over the frames that
    render the same query array (frames are grouped by the identity of their f)."""
    cfg = cfg or LossConfig()
    s0 = scenes[0]
    projs = [project_scene(s) for s in scenes]
    Qs = [render_frame(p, s.f, s.camera)[0] for p, s in zip(projs, scenes)]
    Q = np.concatenate(Qs)
    F = np.concatenate([s.F for s in scenes])
    mask = np.concatenate([s.mask for s in scenes])
    S, A, Fh = decode(Q, s0.K, s0.V, cfg.c(Q.shape[1]))
    parts, _ = loss(Fh, F, mask, s0.V, s0.V0, cfg, Q.shape[1])
    dQ, dK, dV = backward(Q, s0.K, s0.V, s0.V0, A, Fh, F, mask, cfg)
    df = {}
    off = 0
    for p, s in zip(projs, scenes):
        n = s.camera.n_pixels
        g = render_frame_bwd(p, dQ[off:off + n], s.camera, s.n, Q.shape[1])
        df[id(s.f)] = df.get(id(s.f), 0.0) + g
        off += n
    return dict(Q=Q, loss=parts, dK=dK, dV=dV, dQ=dQ, df=df)
