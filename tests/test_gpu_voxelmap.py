"""Parity of the voxel-hashed map (latentam_map_*) with the oracle of oracle/voxelmap.py: every
decision is integer arithmetic or a float32 comparison rounded the same way on both sides, and
every attribute a copy, so the store, the slot table, the indices and the local map are compared
bit for bit; the building workload (2M Gaussians) is checked against a brute-force radius
filter."""
import numpy as np
import pytest

from oracle import voxelmap as vm
from workloads import building_gaussians

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2602_12314_gb300 import api as _api
    return _api


@pytest.fixture(scope="module")
def ctx(api):
    c = api.Context(0)
    yield c
    c.close()


def _gauss(rng, means, d):
    n = len(means)
    return dict(means=np.asarray(means, np.float32), quats=rng.normal(size=(n, 4)).astype(np.float32),
                scales=rng.uniform(0.01, 0.02, size=(n, 3)).astype(np.float32),
                opacities=rng.uniform(0.2, 0.9, size=n).astype(np.float32), f=rng.normal(size=(n, d)).astype(np.float32))


def _args(g):
    return [g[k] for k in ("means", "quats", "scales", "opacities", "f")]


def _np(t):
    return t.cpu().numpy()


def _same_store(gm, om):
    st = gm.global_store()
    arr = om.arrays()
    assert st["means"].shape[0] == om.count
    for k in vm.FIELDS:
        np.testing.assert_array_equal(_np(st[k]), arr[k], err_msg=k)
    np.testing.assert_array_equal(_np(st["table"]), om.table.astype(np.int32))


def test_insert_matches_oracle_with_collisions(api, ctx):
    """A 4096-slot table under 3,000 Gaussians in a 1 m cube (1 cm voxels): many collisions,
    repeated voxels inside a batch, a second batch and a batch of exact duplicates."""
    rng = np.random.default_rng(0)
    d = 8
    gm = api.VoxelMap(ctx, d, table_log2=12, voxel_size=0.01, capacity=100)  # grows
    om = vm.GlobalMap(d, 12, 0.01)
    b1 = _gauss(rng, rng.uniform(-0.5, 0.5, size=(2000, 3)), d)
    b1["means"][1000:1100] = b1["means"][900:1000] + 0.001  # same voxels within the batch
    b2 = _gauss(rng, rng.uniform(-0.5, 0.5, size=(1000, 3)), d)
    for b in (b1, b2, b1):
        idx, n = gm.insert(*_args(b))
        oi = om.insert(b)
        np.testing.assert_array_equal(_np(idx), oi.astype(np.int32))
        assert n == int((oi >= 0).sum())
        _same_store(gm, om)
    assert om.count < 3000  # collisions and duplicates were rejected
    gm.close()


@pytest.mark.parametrize("host_store", [False, True])
def test_sync_sequence_matches_oracle(api, ctx, host_store):
    """Insert 5,000 Gaussians in a 10 m box, then walk the camera: after each synchronisation
    the local map and the store equal the oracle's; between them the local queries change (what
    an optimiser would do), new local Gaussians appear, and the moments travel with their rows."""
    rng = np.random.default_rng(1)
    d = 16
    gm = api.VoxelMap(ctx, d, table_log2=16, voxel_size=0.05, capacity=1000, host_store=host_store)
    om = vm.GlobalMap(d, 16, 0.05)
    g0 = _gauss(rng, rng.uniform(-5, 5, size=(5000, 3)), d)
    gm.insert(*_args(g0))
    om.insert(g0)
    olocal = {k: [] for k in vm.FIELDS}
    olocal["gidx"] = []
    for step, c in enumerate(([0, 0, 0], [1.0, 0.5, 0], [2.5, 1.0, 0.2], [-1, -1, 0], [4, 4, 0])):
        if step:
            loc = gm.local()
            loc["f"] += 1.0  # in place, in the map's memory
            loc["m_f"].copy_(torch.arange(loc["m_f"].numel(), device="cuda", dtype=torch.float32).view_as(loc["m_f"]))
            olocal["f"] = [np.array(x, np.float32) + np.float32(1.0) for x in olocal["f"]]
            marker = {int(gi): _np(loc["m_f"][i]) for i, gi in enumerate(_np(loc["gidx"])) if gi >= 0}
            new = _gauss(rng, np.asarray(c, np.float32) + rng.uniform(-0.5, 0.5, size=(30, 3)), d)
            gm.add_local(*_args(new))
            for k in vm.FIELDS:
                olocal[k] += [np.array(x, np.float32) for x in new[k]]
            olocal["gidx"] += [-1] * 30
        loc = gm.sync(c, 2.0)
        olocal = om.sync(olocal, np.asarray(c, np.float32), 2.0)
        n = len(olocal["gidx"])
        assert loc["means"].shape[0] == n
        np.testing.assert_array_equal(_np(loc["gidx"]), np.array(olocal["gidx"], np.int32))
        for k in vm.FIELDS:
            want = np.array(olocal[k], np.float32).reshape(_np(loc[k]).shape)
            np.testing.assert_array_equal(_np(loc[k]), want, err_msg=k)
        _same_store(gm, om)
        if step:
            gidx = _np(loc["gidx"])
            for i, gi in enumerate(gidx):  # kept rows carry their moments, appended rows start at 0
                if gi in marker:
                    np.testing.assert_array_equal(_np(loc["m_f"][i]), marker[gi])
                elif gi >= 0:
                    assert float(loc["m_f"][i].abs().max()) == 0.0
    gm.close()


def test_empty_map_and_zero_radius(api, ctx):
    gm = api.VoxelMap(ctx, 4, table_log2=8, voxel_size=0.1)
    loc = gm.sync([0, 0, 0], 1.0)
    assert loc["means"].shape == (0, 3)
    rng = np.random.default_rng(2)
    g = _gauss(rng, [[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]], 4)
    gm.insert(*_args(g))
    loc = gm.sync([0.0, 0.0, 0.0], 0.0)  # only the Gaussian exactly at the centre
    np.testing.assert_array_equal(_np(loc["gidx"]), [0])
    gm.close()


@pytest.mark.parametrize("host_store", [False, True])
def test_building_active_set(api, ctx, host_store):
    """The two-floor building (2M Gaussians, 1 cm voxels, 2^24 slots), with the store in HBM or
    in pinned host memory: the local map around a camera with the 5 m active radius is exactly
    the brute-force radius filter of the store, in index order, each row a copy of its store
    entry."""
    g = building_gaussians(0)
    gm = api.VoxelMap(ctx, 32, table_log2=24, voxel_size=0.01, capacity=1 << 21, host_store=host_store)
    idx, n = gm.insert(*_args(g))
    idx = _np(idx)
    # into an empty table the winners are the first Gaussian of every occupied slot, in input
    # order (the oracle's rule, vectorised: uint64 products wrap like the 64-bit hash)
    v = vm.voxel(g["means"], 0.01).astype(np.uint64)
    h = (v[:, 0] * np.uint64(73856093)) ^ (v[:, 1] * np.uint64(19349663)) ^ (v[:, 2] * np.uint64(83492791))
    slots = (h & np.uint64((1 << 24) - 1)).astype(np.int64)
    assert all(int(slots[i]) == vm.hash_slot(vm.voxel(g["means"][i], 0.01), 24) for i in range(0, 2_000_000, 99_991))
    _, first = np.unique(slots, return_index=True)
    want = np.full(len(slots), -1, np.int64)
    want[np.sort(first)] = np.arange(first.size)
    np.testing.assert_array_equal(idx, want.astype(np.int32))
    assert n == first.size
    st = gm.global_store()
    means = _np(st["means"])
    np.testing.assert_array_equal(means, g["means"][idx >= 0])
    for c in ([5.0, 7.5, 1.5], [15.0, 2.5, 4.5]):
        loc = gm.sync(c, 5.0)
        want = np.flatnonzero(vm.in_radius(means, np.asarray(c, np.float32), 5.0))
        np.testing.assert_array_equal(_np(loc["gidx"]), want.astype(np.int32))
        np.testing.assert_array_equal(_np(loc["f"]), _np(st["f"])[want])
    gm.close()


def test_latent_map_optimises_the_active_local_map(api, ctx):
    """LatentMap over a voxel map (Sec. III-E with Algorithm 1): each keyframe synchronises the
    map around its camera, the local Gaussians' queries are optimised in place, and the next
    synchronisation writes them back to the store; Gaussians never in an active set keep their
    queries."""
    from workloads import room_views, sam_masks
    views = room_views(9, n_views=3, n=40_000, width=96, height=72, fx=78.75)
    s = views[0]
    vmap = api.VoxelMap(ctx, s.d, table_log2=20, voxel_size=0.01)
    _, n = vmap.insert(s.means, s.quats, s.scales, s.opacities, s.f)
    f0 = vmap.global_store()["f"].clone()
    m = api.LatentMap(ctx, s, B=1, voxel_map=vmap, radius=4.0)
    seen = set()
    for v in views:
        r = m.add_keyframe(v.camera, masks=sam_masks(v, cell=(24, 18)))
        assert np.isfinite(r["stage1"]["total"]) and np.isfinite(r["stage2"]["total"])
        loc = vmap.local()
        centre = -v.camera.R.astype(np.float64).T @ v.camera.t.astype(np.float64)
        want = np.flatnonzero(vm.in_radius(_np(vmap.global_store()["means"]), centre.astype(np.float32), 4.0))
        np.testing.assert_array_equal(np.sort(_np(loc["gidx"])), want.astype(np.int32))
        seen |= set(want.tolist())
    vmap.sync([100.0, 100.0, 100.0], 0.1)  # write everything back, keep nothing local
    f1 = _np(vmap.global_store()["f"])
    changed = np.flatnonzero(np.abs(f1 - _np(f0)).max(axis=1) > 0)
    # the rendered ones among the active Gaussians learned (the rest of the sphere is out of view)
    assert len(changed) > 1000 and set(changed.tolist()) <= seen
    vmap.close()
