"""ctypes view of include/latentam.h: struct layouts, status codes and the loaded library.

Argument marshalling only; every step of the computation runs in liblatentam.so.  There is
no fallback: if the library is missing or fails to load, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

OK = 0
ERR_INVALID_ARG = -1
ERR_UNSUPPORTED_SHAPE = -2
ERR_OUT_OF_MEMORY = -3
ERR_CUDA = -4
ERR_CAPACITY = -5
ERR_TIMEOUT = -6
ERR_NOT_FINITE = -7
_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "UNSUPPORTED_SHAPE", -3: "OUT_OF_MEMORY", -4: "CUDA", -5: "CAPACITY",
          -6: "TIMEOUT", -7: "NOT_FINITE"}

ABI_VERSION = 3

PREC_FP32 = 0
PREC_BF16 = 1
PREC_FP8 = 2
PREC_FP32_FMA = 3
DTYPE_F32 = 0
DTYPE_BF16 = 1
LOSS_PARTS = 5
TILE = 16
STAGES = ("project", "sort", "render_fwd", "decode", "render_bwd", "adam")

P = ctypes.c_void_p
F32 = ctypes.c_float
I32 = ctypes.c_int32
I64 = ctypes.c_int64


class LatentamError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"latentam {_NAMES.get(status, status)}: {msg}")
        self.status = status


class Camera(ctypes.Structure):
    _fields_ = [("R", F32 * 9), ("t", F32 * 3), ("fx", F32), ("fy", F32), ("cx", F32), ("cy", F32),
                ("z_near", F32), ("width", I32), ("height", I32)]


class Gaussians(ctypes.Structure):
    _fields_ = [("n", I32), ("means", P), ("quats", P), ("scales", P), ("opacities", P)]


class Projected(ctypes.Structure):
    _fields_ = [("xy", P), ("conic_opacity", P), ("depth", P), ("rect", P), ("tiles_touched", P)]


class Bins(ctypes.Structure):
    _fields_ = [("pair_ids", P), ("capacity", I64), ("tile_ranges", P), ("num_pairs", I64)]


class LossCfg(ctypes.Structure):
    _fields_ = [("lambda_f", F32), ("lambda_cos", F32), ("lambda_2", F32), ("lambda_D", F32), ("delta", F32),
                ("logit_scale", F32)]


class AdamCfg(ctypes.Structure):
    _fields_ = [("lr_f", F32), ("lr_dict", F32), ("beta1", F32), ("beta2", F32), ("eps", F32), ("step", I32)]


class Frame(ctypes.Structure):
    _fields_ = [("gaussians", Gaussians), ("camera", Camera), ("F", P), ("F_dtype", I32), ("mask", P),
                ("mask_offsets", P), ("mask_pixels", P), ("n_mask_entries", I64), ("n_masks", I32)]


class Params(ctypes.Structure):
    _fields_ = [("f", P), ("K", P), ("V", P), ("V0", P), ("m_f", P), ("v_f", P), ("m_K", P), ("v_K", P),
                ("m_V", P), ("v_V", P), ("d", I32), ("M", I32), ("D", I32), ("tau", F32)]


class BatchFrame(ctypes.Structure):
    _fields_ = [("gaussians", Gaussians), ("camera", Camera), ("f", P), ("m_f", P), ("v_f", P),
                ("mask_offsets", P), ("mask_pixels", P), ("n_mask_entries", I64), ("n_masks", I32)]


class ImageCfg(ctypes.Structure):
    _fields_ = [("lambda_rgb", F32), ("lambda_I1", F32), ("lambda_I2", F32), ("lambda_d", F32)]


FULL_LOSS_PARTS = 10


class MapLocal(ctypes.Structure):
    _fields_ = [("means", P), ("quats", P), ("scales", P), ("opacities", P), ("f", P), ("m_f", P), ("v_f", P),
                ("gidx", P), ("count", I64)]


class MapGlobal(ctypes.Structure):
    _fields_ = [("means", P), ("quats", P), ("scales", P), ("opacities", P), ("f", P), ("table", P),
                ("count", I64), ("table_size", I64)]


class Dictionary(ctypes.Structure):
    _fields_ = [("K", P), ("V", P), ("V0", P), ("m_K", P), ("v_K", P), ("m_V", P), ("v_V", P), ("d", I32),
                ("M", I32), ("D", I32), ("tau", F32)]


class TuneChoice(ctypes.Structure):
    _fields_ = [("n", I64), ("M", I32), ("D", I32), ("reduction", I32), ("tile", I32), ("split", I32),
                ("ms", F32)]


MAX_BATCH = 32

_SIGS = {
    "latentam_version": ([], I32),
    "latentam_launch_count": ([], I64),
    "latentam_last_error": ([], ctypes.c_char_p),
    "latentam_num_tiles": ([ctypes.POINTER(Camera)], I32),
    "latentam_ctx_create": ([I32, ctypes.POINTER(P)], I32),
    "latentam_ctx_destroy": ([P], I32),
    "latentam_profile_enable": ([P, I32], I32),
    "latentam_graphs_enable": ([P, I32], I32),
    "latentam_autotune_enable": ([P, I32], I32),
    "latentam_autotune_query": ([P, I32, ctypes.POINTER(TuneChoice), ctypes.POINTER(I32)], I32),
    "latentam_test_wait_timeout": ([P, I32], I32),
    "latentam_profile_read": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64), I32], I32),
    "latentam_project": ([P, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), ctypes.POINTER(Projected), P], I32),
    "latentam_sort": ([P, I32, ctypes.POINTER(Projected), ctypes.POINTER(Camera), ctypes.POINTER(Bins), P], I32),
    "latentam_render_fwd": ([P, I32, ctypes.POINTER(Projected), ctypes.POINTER(Camera), ctypes.POINTER(Bins), P, I32,
                             P, P, P, P], I32),
    "latentam_render_bwd": ([P, I32, ctypes.POINTER(Projected), ctypes.POINTER(Camera), ctypes.POINTER(Bins), P, P,
                             I32, P, P], I32),
    "latentam_decode_fwd": ([P, P, I64, I32, P, P, I32, I32, F32, I32, P, P, P], I32),
    "latentam_decode_loss_bwd": ([P, P, I64, I32, P, P, P, I32, I32, P, I32, P, ctypes.POINTER(LossCfg), I32, P, P,
                                  P, P, P], I32),
    "latentam_decode_fwd_paper": ([P, P, I64, I32, P, P, I32, I32, F32, I32, P, P, P], I32),
    "latentam_decode_loss_bwd_paper": ([P, P, I64, I32, P, P, P, I32, I32, F32, P, I32, P, ctypes.POINTER(LossCfg), I32,
                                        P, P, P, P, P], I32),
    "latentam_decode_loss_bwd_noalloc": ([P, P, I64, I32, P, P, P, I32, I32, P, I32, P, ctypes.POINTER(LossCfg), P, P,
                                          P, P, P], I32),
    "latentam_backward": ([P, I32, ctypes.POINTER(Projected), ctypes.POINTER(Camera), ctypes.POINTER(Bins), P, P,
                           I32, P, P, P, I32, I32, P, I32, P, ctypes.POINTER(LossCfg), I32, P, P, P, P, P, P], I32),
    "latentam_pool_queries": ([P, P, I64, I32, P, P, I64, I32, P, P], I32),
    "latentam_pool_queries_bwd": ([P, P, I32, I32, P, P, I64, I64, P, P], I32),
    "latentam_stream_kmeans": ([P, P, I64, I32, P, P, I32, I32, I32, P, P, I32, P, P, P, P, P], I32),
    "latentam_backward_full": ([P, ctypes.POINTER(Gaussians), P, P, I32, ctypes.POINTER(Camera), P, P, P, I32, I32,
                                P, I32, P, P, P, ctypes.POINTER(LossCfg), ctypes.POINTER(ImageCfg), I32, P, P, P, P,
                                P, P, P, P, P, P], I32),
    "latentam_map_create": ([P, I32, I32, F32, I64, I32, ctypes.POINTER(P)], I32),
    "latentam_map_destroy": ([P], I32),
    "latentam_map_insert": ([P, P, ctypes.POINTER(Gaussians), P, P, ctypes.POINTER(I64), P], I32),
    "latentam_map_add_local": ([P, P, ctypes.POINTER(Gaussians), P, P], I32),
    "latentam_map_sync": ([P, P, ctypes.POINTER(F32), F32, ctypes.POINTER(MapLocal), P], I32),
    "latentam_map_local_view": ([P, ctypes.POINTER(MapLocal)], I32),
    "latentam_map_global_view": ([P, ctypes.POINTER(MapGlobal)], I32),
    "latentam_adam": ([P, I32, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                       ctypes.POINTER(I64), ctypes.POINTER(F32), ctypes.POINTER(AdamCfg), P], I32),
    "latentam_step": ([P, ctypes.POINTER(Frame), ctypes.POINTER(Params), ctypes.POINTER(LossCfg),
                       ctypes.POINTER(AdamCfg), I32, I32, I32, ctypes.POINTER(ctypes.c_double), P], I32),
    "latentam_step_batch": ([P, ctypes.POINTER(BatchFrame), I32, P, I32, P, ctypes.POINTER(Dictionary),
                             ctypes.POINTER(LossCfg), ctypes.POINTER(AdamCfg), I32, I32, I32,
                             ctypes.POINTER(ctypes.c_double), P], I32),
}

EXPORTED = tuple(_SIGS)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load liblatentam.so (building it first only when asked)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with paper_2602_12314_gb300.build.build() "
                                   "(there is no CPU fallback)")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            if lib.latentam_version() != ABI_VERSION:
                raise RuntimeError("liblatentam.so ABI version mismatch")
            _lib = lib
    return _lib


def check(status: int):
    if status != OK:
        raise LatentamError(status, _lib.latentam_last_error().decode(errors="replace"))
