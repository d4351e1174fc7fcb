"""GB300-native (sm_103a) latent-feature optimisation step of LatentAM (arxiv 2602.12314).

The computation lives in liblatentam.so (include/latentam.h); this package is its build
script, its ctypes binding (``api``) and autograd wrappers (``autograd``).
"""
from . import build  # noqa: F401

__all__ = ["api", "autograd", "build"]


def __getattr__(name):
    if name in ("api", "autograd"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
