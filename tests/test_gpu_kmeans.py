"""Parity of the streaming K-means dictionary update (latentam_stream_kmeans) with the FP64 oracle
of oracle/kmeans.py.

Two kinds of check, because every decision of K-means is an argmin of float distances:
  * exact comparison with the oracle from the same state, on inputs whose decisions are far
    from ties (each case asserts that the oracle's smallest decision gap is far above float32
    rounding): assignments and weights bit-exact, centres within a relative 1e-5 per row;
  * replay validation on realistic inputs (noisy per-pixel and per-mask targets of one room,
    where some row always lies almost exactly between two centres and either choice is
    correct): the GPU path is deterministic, so a run with one iteration fewer yields the
    centres each final decision was taken against; every final assignment must be within
    1e-4 (relative) of the nearest distance in float64, every centre the float64 weighted mean
    of its rows or points (relative 1e-5), and every weight the exact count or weight sum."""
import numpy as np
import pytest

from oracle import kmeans as km
from workloads import room_scene, room_views, sam_masks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS_DECISION = 1e-4


@pytest.fixture(scope="module")
def api():
    from paper_2602_12314_gb300 import api as _api
    return _api


@pytest.fixture(scope="module")
def ctx(api):
    c = api.Context(0)
    yield c
    c.close()


def _dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _rel_rows(a, b, floor=1e-6):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), floor)


def _gpu(api, ctx, F, valid, C, W, init, il, ig):
    Cd, Wd = _dev(C), _dev(W)
    vd = _dev(valid, torch.uint8) if valid is not None else None
    mC, mW, ma, pa = api.stream_kmeans(ctx, _dev(F), Cd, Wd, init, valid=vd, iters_local=il, iters_global=ig,
                                       want_micro=True)
    return dict(C=Cd.cpu().numpy(), W=Wd.cpu().numpy(), mC=mC.cpu().numpy(), mW=mW.cpu().numpy(),
                ma=ma.cpu().numpy(), pa=pa.cpu().numpy())


def _exact(api, ctx, F, valid, C, W, init, il, ig, gap_floor=1e-3):
    g = _gpu(api, ctx, F, valid, C, W, init, il, ig)
    o = km.stream_kmeans(F, valid, C.astype(np.float64), W.astype(np.float64), init, il, ig)
    assert o["min_gap"] > gap_floor, o["min_gap"]
    np.testing.assert_array_equal(g["ma"], o["micro_assign"])
    np.testing.assert_array_equal(g["mW"], o["micro_weights"])
    live = o["micro_weights"] > 0
    if live.any():
        assert _rel_rows(g["mC"][live].astype(np.float64), o["micro_centres"][live]).max() <= 1e-5
    np.testing.assert_array_equal(g["W"], o["weights"])
    assert _rel_rows(g["C"].astype(np.float64), o["centres"]).max() <= 1e-5
    return g["C"], g["W"]


def _eps_optimal(X, Cand, active, chosen):
    d = km.sq_dist(X, Cand)
    if active is not None:
        d[:, ~active] = np.inf
    best = d.min(axis=1)
    got = d[np.arange(X.shape[0]), chosen]
    assert np.all(got <= best + EPS_DECISION * (1.0 + best)), float((got - best).max())


def _replay(api, ctx, F, valid, C, W, init, il, ig):
    """Validates one call on realistic inputs (see the module docstring); returns its output."""
    g = _gpu(api, ctx, F, valid, C, W, init, il, ig)
    F64 = F.astype(np.float64)
    rows = np.arange(F.shape[0]) if valid is None else np.flatnonzero(valid)
    # local phase: the last assignment against the centres one iteration earlier
    prev = F64[np.asarray(init)] if il == 1 else _gpu(api, ctx, F, valid, C, W, init, il - 1, ig)["mC"]
    assert np.all(g["ma"][np.setdiff1d(np.arange(F.shape[0]), rows)] == -1)
    _eps_optimal(F64[rows], prev.astype(np.float64), None, g["ma"][rows])
    k = len(init)
    np.testing.assert_array_equal(g["mW"], np.bincount(g["ma"][rows], minlength=k))
    for c in range(k):
        if g["mW"][c] > 0:
            ref = F64[g["ma"] == c].mean(axis=0)
            assert np.linalg.norm(g["mC"][c] - ref) <= 1e-5 * np.linalg.norm(ref)
    # global phase: the merged points and active slots by the merge rule from the GPU's micro-clusters
    used = np.flatnonzero(W > 0)
    live = np.flatnonzero(g["mW"] > 0)
    P = np.concatenate([C[used], g["mC"][live]]).astype(np.float64)
    pw = np.concatenate([W[used], g["mW"][live]]).astype(np.float64)
    start = C.astype(np.float64).copy()
    active = W > 0
    for slot, c in zip(np.flatnonzero(W <= 0), sorted(live.tolist(), key=lambda c: (-g["mW"][c], c))):
        start[slot] = g["mC"][c]
        active[slot] = True
    pa = g["pa"]
    assert np.all(pa[len(P):] == -1)
    pa = pa[:len(P)]
    cprev = start if ig == 1 else _gpu(api, ctx, F, valid, C, W, init, il, ig - 1)["C"].astype(np.float64)
    _eps_optimal(P, cprev, active, pa)
    for s in range(C.shape[0]):
        members = pa == s
        if not active[s]:
            assert g["W"][s] == W[s] == 0 and np.array_equal(g["C"][s], C[s])
            continue
        assert g["W"][s] == pw[members].sum()
        if members.any():
            ref = (pw[members, None] * P[members]).sum(axis=0) / pw[members].sum()
            assert np.linalg.norm(g["C"][s] - ref) <= 1e-5 * max(np.linalg.norm(ref), 1e-6)
        else:
            np.testing.assert_allclose(g["C"][s], cprev[s], rtol=1e-6)
    # repeated calls are bit-identical
    again = _gpu(api, ctx, F, valid, C, W, init, il, ig)
    for key in ("C", "W", "mC", "ma", "pa"):
        np.testing.assert_array_equal(again[key], g[key])
    return g


def _blobs(rng, E, shown, per=(3, 20), noise=0.01):
    """Masks of the shown embeddings: a few near-duplicates of each, l2-normalised."""
    rows, lab = [], []
    for i in shown:
        m = int(rng.integers(*per))
        x = E[i] + rng.normal(0, noise, size=(m, E.shape[1]))
        rows.append(x / np.linalg.norm(x, axis=1, keepdims=True))
        lab += [i] * m
    F = np.concatenate(rows).astype(np.float32)
    perm = rng.permutation(F.shape[0])
    return F[perm], np.array(lab)[perm]


def test_exact_stream_fills_then_merges(api, ctx):
    """Ten semantic embeddings in K = 10 slots: two keyframes of five new ones fill the
    dictionary, eight more keyframes each show five of the ten and merge into their slots."""
    rng = np.random.default_rng(0)
    D, K = 512, 10
    E = rng.normal(size=(10, D))
    E /= np.linalg.norm(E, axis=1, keepdims=True)
    C = rng.normal(size=(K, D)).astype(np.float32)
    W = np.zeros(K, np.float32)
    total = 0
    for t in range(10):
        shown = list(range(5 * t, 5 * t + 5)) if t < 2 else sorted(rng.choice(10, size=5, replace=False))
        F, lab = _blobs(rng, E, shown)
        valid = (rng.uniform(size=F.shape[0]) > 0.1).astype(np.uint8)
        valid[[int(np.flatnonzero(lab == i)[0]) for i in shown]] = 1
        init = np.array([int(np.flatnonzero(lab == i)[0]) for i in shown], np.int32)
        C, W = _exact(api, ctx, F, valid, C, W, init, 5, 5)
        total += int(valid.sum())
    assert (W > 0).all() and W.sum() == total


def test_replay_stream_of_room_keyframes(api, ctx):
    """Twenty keyframes of one room's SAM-style mask targets (D = 512) into K = 64 slots with
    5 micro-clusters each: the dictionary fills in thirteen keyframes, then every keyframe
    merges into atoms that repeat the room's segments (near-ties are common)."""
    views = room_views(3, n_views=20, n=2000, width=160, height=120, fx=131.25)
    rng = np.random.default_rng(0)
    K, D = 64, views[0].D
    C = rng.normal(size=(K, D)).astype(np.float32)
    W = np.zeros(K, np.float32)
    total = 0
    for v in views:
        ms = sam_masks(v, cell=(20, 15), seed=1)
        rows = np.flatnonzero(ms.valid)
        init = rng.choice(rows, size=5, replace=False).astype(np.int32)
        g = _replay(api, ctx, ms.F, ms.valid, C, W, init, 10, 10)
        C, W = g["C"], g["W"]
        total += int(ms.valid.sum())
    assert (W > 0).sum() >= 60 and W.sum() == total


@pytest.mark.parametrize("D,k,K", [(512, 8, 128), (768, 32, 301), (256, 3, 17)])
def test_replay_per_pixel_features(api, ctx, D, k, K):
    """Per-pixel targets (19,200 rows) into a half-occupied dictionary; ragged K, D = 768."""
    s = room_scene(7, n=2000, D=D, width=160, height=120, fx=131.25)
    rng = np.random.default_rng(D + k)
    rows = np.flatnonzero(s.mask)
    C = (s.F[rng.choice(rows, size=K)] + rng.normal(0, 0.05, size=(K, D))).astype(np.float32)
    W = np.where(rng.uniform(size=K) < 0.5, rng.integers(1, 50, size=K), 0).astype(np.float32)
    init = rng.choice(rows, size=k, replace=False).astype(np.int32)
    _replay(api, ctx, s.F, s.mask, C, W, init, 6, 6)


def test_edge_cases(api, ctx):
    rng = np.random.default_rng(3)
    D = 64
    # one row, one micro-cluster, an empty dictionary of one slot
    F = rng.normal(size=(1, D)).astype(np.float32)
    C, W = _exact(api, ctx, F, None, np.zeros((1, D), np.float32), np.zeros(1, np.float32),
                  np.array([0], np.int32), 1, 1)
    np.testing.assert_allclose(C[0], F[0], rtol=1e-6)
    assert W[0] == 1
    # every row invalid: no live micro-cluster, the dictionary is unchanged
    F = rng.normal(size=(40, D)).astype(np.float32)
    C0 = rng.normal(size=(8, D)).astype(np.float32) * 5
    W0 = np.array([1, 2, 0, 3, 0, 0, 4, 1], np.float32)
    C, W = _exact(api, ctx, F, np.zeros(40, np.uint8), C0, W0, np.array([0, 1], np.int32), 3, 3)
    np.testing.assert_array_equal(W, W0)
    np.testing.assert_allclose(C, C0, rtol=1e-6)


def test_rejects_unsupported_shapes(api, ctx):
    from paper_2602_12314_gb300 import _lib as L
    F = torch.zeros((10, 64), device="cuda")
    C, W = torch.zeros((4, 64), device="cuda"), torch.zeros(4, device="cuda")
    for init in (np.arange(33) % 10, np.arange(11) % 10):  # k > 32, k > n
        with pytest.raises(L.LatentamError) as e:
            api.stream_kmeans(ctx, F, C, W, init)
        assert e.value.status == L.ERR_UNSUPPORTED_SHAPE
    with pytest.raises(L.LatentamError) as e:  # D not a multiple of 4
        api.stream_kmeans(ctx, torch.zeros((10, 30), device="cuda"), torch.zeros((4, 30), device="cuda"), W, [0])
    assert e.value.status == L.ERR_UNSUPPORTED_SHAPE


def test_full_size_per_pixel(api, ctx):
    """640x480 per-pixel targets (307,200 rows, D = 512), 5 micro-clusters into K = 256 slots
    of which 100 are occupied, replay-validated."""
    s = room_scene(0, n=2000)
    rng = np.random.default_rng(11)
    rows = np.flatnonzero(s.mask)
    init = rng.choice(rows, size=5, replace=False).astype(np.int32)
    K = 256
    C = rng.normal(size=(K, s.D)).astype(np.float32)
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    W = np.zeros(K, np.float32)
    W[:100] = rng.integers(1, 1000, size=100)
    _replay(api, ctx, s.F, s.mask, C, W, init, 4, 4)
