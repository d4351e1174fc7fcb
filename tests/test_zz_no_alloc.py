"""latentam_decode_loss_bwd_noalloc: the decode + loss + backward for callers that cannot
allocate device memory while the step runs (for instance a real-time loop whose device
memory was carved up once at start-up by another runtime's allocator, or a caller that
cannot absorb the device-wide synchronisation cudaMalloc/cudaFree may cause).  Its scratch
is a static device array inside the library instead of the context's growable workspace.

Called through the C ABI twice in a row, on different inputs, and checked each time against
latentam_decode_loss_bwd and against the FP64 oracle at the FP32 tolerances the other GPU
tests use, over the query widths, dictionary sizes (including one that is not a multiple of
the kernels' 128-atom chunks, and the largest, whose rows need 128 KiB of shared memory) and
target types the kernels are instantiated for, without a mask and without dQ; a fresh
context's first call must not change the free device memory; an oversized call must be
refused with a clear error.  This file is named to be collected last, so that a run stopping
at the first failure has already run every other test; it creates its own contexts and
inputs, so it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle

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


def _inputs(seed, n, d=32, M=256, D=512, mask_drop=0.2, target=torch.float32):
    rng = np.random.default_rng(seed)
    dev = "cuda"
    Q = torch.tensor(rng.normal(size=(n, d)), dtype=torch.float32, device=dev)
    K = torch.tensor(rng.normal(size=(M, d)) / np.sqrt(d), dtype=torch.float32, device=dev)
    V = torch.tensor(rng.normal(size=(M, D)) / np.sqrt(d), dtype=torch.float32, device=dev)
    V0 = (V + 0.05 * torch.tensor(rng.normal(size=(M, D)), dtype=torch.float32, device=dev)
          * (torch.arange(M, device=dev) % 2)[:, None]).contiguous()
    F = rng.normal(size=(n, D))
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    F = torch.tensor(F, dtype=torch.float32, device=dev).to(target)
    mask = torch.tensor(rng.uniform(size=n) >= mask_drop, dtype=torch.uint8, device=dev) if mask_drop else None
    return Q, K, V, V0, F, mask


def _oracle(args):
    Q, K, V, V0, F, mask = (None if x is None else x.float().cpu().numpy() for x in args)
    n, d = Q.shape
    mask = np.ones(n, np.uint8) if mask is None else mask.astype(np.uint8)
    cfg = oracle.LossConfig()
    _, A, Fo = oracle.decode(Q, K, V, cfg.c(d))
    parts, _ = oracle.loss(Fo, F, mask, V, V0, cfg, d)
    dQ, dK, dV = oracle.backward(Q, K, V, V0, A, Fo, F, mask, cfg)
    return np.array([parts["cos"], parts["l2"], parts["tr"], parts["total"], parts["n_valid"]]), dQ, dK, dV


def _rel(g, w):
    g, w = np.asarray(g, np.float64), np.asarray(w, np.float64)
    return float(np.linalg.norm(g - w) / np.linalg.norm(w))


def _compare(got, want, oracle_want):
    gp, gq, gk, gv = got
    wp, wq, wk, wv = want
    torch.testing.assert_close(gp, wp, rtol=REL_LOSS, atol=1e-12)
    op, oq, ok_, ov = oracle_want
    np.testing.assert_allclose(gp.cpu().numpy(), op, rtol=REL_LOSS, atol=1e-12)
    for g, w, o in ((gq, wq, oq), (gk, wk, ok_), (gv, wv, ov)):
        if g is None:
            assert w is None
            continue
        assert _rel(g.cpu().numpy(), w.cpu().numpy()) <= REL_G
        assert _rel(g.cpu().numpy(), o) <= REL_G


@pytest.mark.parametrize("d,M,target", [(32, 256, "f32"), (16, 96, "f32"), (64, 1024, "f32"), (32, 96, "bf16"),
                                        (16, 1024, "bf16"), (64, 256, "bf16")])
def test_noalloc_matches_workspace_entry_point_twice(api, ctx, d, M, target):
    tdt = torch.float32 if target == "f32" else torch.bfloat16
    n_big = 1500 if M <= 256 else 300
    for seed, n in ((1, n_big), (2, n_big // 2 + 37)):
        args = _inputs(seed + d + M, n, d=d, M=M, target=tdt)
        want = api.decode_loss_bwd(ctx, *args, api.LossConfig(), api.FP32)
        got = api.decode_loss_bwd_noalloc(ctx, *args, api.LossConfig())
        torch.cuda.synchronize()
        _compare(got, want, _oracle(args))


def test_noalloc_without_mask_and_without_dq(api, ctx):
    args = _inputs(5, 700, mask_drop=0.0)
    assert args[5] is None
    want = api.decode_loss_bwd(ctx, *args, api.LossConfig(), api.FP32, need_dQ=False)
    parts = torch.empty((5,), dtype=torch.float64, device="cuda")
    dK = torch.empty((256, 32), device="cuda")
    dV = torch.empty((256, 512), device="cuda")
    for _ in range(2):
        got = api.decode_loss_bwd_noalloc(ctx, *args, api.LossConfig(), out=(parts, None, dK, dV))
        torch.cuda.synchronize()
        _compare(got, want, _oracle(args))


def test_noalloc_first_call_on_fresh_context_allocates_nothing(api):
    args = _inputs(3, 1024)
    with api.Context(0) as fresh:
        out = (torch.empty((5,), dtype=torch.float64, device="cuda"), torch.empty((1024, 32), device="cuda"),
               torch.empty((256, 32), device="cuda"), torch.empty((256, 512), device="cuda"))
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        api.decode_loss_bwd_noalloc(fresh, *args, api.LossConfig(), out=out)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free0 == free1
        api.decode_loss_bwd_noalloc(fresh, *args, api.LossConfig(), out=out)
        torch.cuda.synchronize()
        free2, _ = torch.cuda.mem_get_info()
        assert free0 == free2
        want = api.decode_loss_bwd(fresh, *args, api.LossConfig(), api.FP32)
        _compare(out, want, _oracle(args))


def test_noalloc_refuses_oversized_calls(api, ctx):
    from paper_2602_12314_gb300 import _lib as L
    args = _inputs(4, 8192)
    with pytest.raises(L.LatentamError) as e:
        api.decode_loss_bwd_noalloc(ctx, *args, api.LossConfig())
    assert e.value.status == L.ERR_UNSUPPORTED_SHAPE
    assert "static scratch" in str(e.value)
