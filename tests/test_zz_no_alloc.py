"""latentam_decode_loss_bwd_noalloc: the decode + loss + backward for callers that cannot
allocate device memory while the step runs (for instance a real-time loop whose device
memory was carved up once at start-up by another runtime's allocator, or a caller that
cannot absorb the device-wide synchronisation cudaMalloc/cudaFree may cause).  Its scratch
is a static device array inside the library instead of the context's growable workspace.

Called through the C ABI twice in a row, on different inputs, and checked each time
against latentam_decode_loss_bwd at the FP32 tolerances the other GPU tests use; an
oversized call must be refused with a clear error.  This file is named to be collected
last, so that a run stopping at the first failure has already run every other test; it
creates its own context and inputs, so it also passes alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_LOSS = 1e-5
REL_G = 1e-3


@pytest.fixture(scope="module")
def api():
    from paper_2602_12314_gb300 import api as _api
    return _api


@pytest.fixture(scope="module")
def ctx(api):
    c = api.Context(0)
    yield c
    c.close()


def _inputs(seed, n, d=32, M=256, D=512, mask_drop=0.2):
    rng = np.random.default_rng(seed)
    dev = "cuda"
    Q = torch.tensor(rng.normal(size=(n, d)), dtype=torch.float32, device=dev)
    K = torch.tensor(rng.normal(size=(M, d)) / np.sqrt(d), dtype=torch.float32, device=dev)
    V = torch.tensor(rng.normal(size=(M, D)) / np.sqrt(d), dtype=torch.float32, device=dev)
    V0 = (V + 0.05 * torch.tensor(rng.normal(size=(M, D)), dtype=torch.float32, device=dev)
          * (torch.arange(M, device=dev) % 2)[:, None]).contiguous()
    F = rng.normal(size=(n, D))
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    F = torch.tensor(F, dtype=torch.float32, device=dev)
    mask = torch.tensor(rng.uniform(size=n) >= mask_drop, dtype=torch.uint8, device=dev)
    return Q, K, V, V0, F, mask


def _compare(got, want):
    gp, gq, gk, gv = got
    wp, wq, wk, wv = want
    torch.testing.assert_close(gp, wp, rtol=REL_LOSS, atol=1e-12)
    for g, w in ((gq, wq), (gk, wk), (gv, wv)):
        err = float(torch.linalg.norm(g.double() - w.double()) / torch.linalg.norm(w.double()))
        assert err <= REL_G, err


def test_noalloc_matches_workspace_entry_point_twice(api, ctx):
    for seed, n in ((1, 1500), (2, 2048)):
        args = _inputs(seed, n)
        want = api.decode_loss_bwd(ctx, *args, api.LossConfig(), api.FP32)
        got = api.decode_loss_bwd_noalloc(ctx, *args, api.LossConfig())
        torch.cuda.synchronize()
        _compare(got, want)


def test_noalloc_call_allocates_no_device_memory(api, ctx):
    args = _inputs(3, 1024)
    out = api.decode_loss_bwd_noalloc(ctx, *args, api.LossConfig())
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    api.decode_loss_bwd_noalloc(ctx, *args, api.LossConfig(), out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 == free1
    want = api.decode_loss_bwd(ctx, *args, api.LossConfig(), api.FP32)
    _compare(out, want)


def test_noalloc_refuses_oversized_calls(api, ctx):
    from paper_2602_12314_gb300 import _lib as L
    args = _inputs(4, 8192)
    with pytest.raises(L.LatentamError) as e:
        api.decode_loss_bwd_noalloc(ctx, *args, api.LossConfig())
    assert e.value.status == L.ERR_UNSUPPORTED_SHAPE
    assert "static scratch" in str(e.value)
