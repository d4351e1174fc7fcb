"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/latentam.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^LATENTAM_API\s+[\w\s\*]+?\b(latentam_\w+)\s*\(", src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2602_12314_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2602_12314_gb300 import _lib
    assert set(_declared()) == set(_lib.EXPORTED)


def test_version_and_tiles_without_gpu(lib):
    from paper_2602_12314_gb300 import _lib
    L = _lib.load()
    assert L.latentam_version() == 3
    cam = _lib.Camera()
    cam.width, cam.height = 640, 480
    assert L.latentam_num_tiles(ctypes.byref(cam)) == 40 * 30
    cam.width, cam.height = 72, 50
    assert L.latentam_num_tiles(ctypes.byref(cam)) == 5 * 4


def test_no_silent_cpu_path():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2602_12314_gb300 import api
    with pytest.raises(RuntimeError):
        api.Context()
