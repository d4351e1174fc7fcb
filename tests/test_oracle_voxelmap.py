"""Pins of the voxel-hashed map oracle (oracle/voxelmap.py): the spatial hash's closed forms on
unit voxels and its 64-bit wrap, floor (not truncation) of negative coordinates, the radius test
against float64 distances away from the boundary, insert-if-free order and collisions on
hand-built cases, and the invariants of a synchronisation sequence."""
import numpy as np
import pytest

from oracle import voxelmap as vm


def test_hash_closed_forms():
    k = 20
    T = 1 << k
    assert vm.hash_slot((0, 0, 0), k) == 0
    assert vm.hash_slot((1, 0, 0), k) == 73856093 % T
    assert vm.hash_slot((0, 1, 0), k) == 19349663 % T
    assert vm.hash_slot((0, 0, 1), k) == 83492791 % T
    assert vm.hash_slot((1, 1, 0), k) == (73856093 ^ 19349663) % T
    # two's complement: -x p has the low bits of 2^64 - x p
    assert vm.hash_slot((-1, 0, 0), k) == (2 ** 64 - 73856093) % T
    assert vm.hash_slot((0, -2, 0), k) == (2 ** 64 - 2 * 19349663) % T
    # products beyond 64 bits wrap
    x = 2 ** 40 + 12345
    assert vm.hash_slot((x, 0, 0), k) == (x * 73856093) % (2 ** 64) % T


def test_voxel_floor_of_float32_quotient():
    s = 0.01
    assert tuple(vm.voxel([0.005, -0.005, -0.0150], s)) == (0, -1, -2)  # floor, not truncation
    rng = np.random.default_rng(0)
    p = rng.uniform(-20, 20, size=(1000, 3)).astype(np.float32)
    v = vm.voxel(p, s)
    q = p.astype(np.float64) / np.float64(np.float32(s))
    away = np.abs(q - np.round(q)) > 1e-3  # off the cell boundaries the float64 floor agrees
    assert np.array_equal(v[away], np.floor(q[away]).astype(np.int64))


def test_radius_test_against_float64_distance():
    rng = np.random.default_rng(1)
    m = rng.uniform(-10, 10, size=(5000, 3)).astype(np.float32)
    c = np.array([1.5, -2.0, 0.3], np.float32)
    r = 4.0
    got = vm.in_radius(m, c, r)
    dist = np.linalg.norm(m.astype(np.float64) - c.astype(np.float64), axis=1)
    clear = np.abs(dist - r) > 1e-4
    assert np.array_equal(got[clear], dist[clear] <= r)
    assert got.sum() > 100 and (~got).sum() > 100


def _gauss(rng, means, d=4):
    n = len(means)
    return dict(means=np.asarray(means, np.float32), quats=rng.normal(size=(n, 4)).astype(np.float32),
                scales=rng.uniform(0.01, 0.02, size=(n, 3)).astype(np.float32),
                opacities=rng.uniform(0.2, 0.9, size=n).astype(np.float32), f=rng.normal(size=(n, d)).astype(np.float32))


def test_insert_if_free_order_and_collisions():
    rng = np.random.default_rng(2)
    k = 4  # 16 slots: collisions are easy to find
    m = vm.GlobalMap(d=4, table_log2=k, voxel_size=0.01)
    # two voxels with the same slot
    a = (0, 0, 0)
    b = next((x, 1, 0) for x in range(1, 1000) if vm.hash_slot((x, 1, 0), k) == vm.hash_slot(a, k))
    pts = [[0.001, 0.002, 0.003],            # voxel a: inserted, index 0
           [0.004, 0.009, 0.001],            # voxel a again: rejected
           [b[0] * 0.01 + 0.005, 0.015, 0.001],  # voxel b, same slot: rejected (collision)
           [0.5, 0.5, 0.5]]                  # elsewhere
    g = _gauss(rng, pts)
    idx = m.insert(g)
    assert idx[0] == 0 and idx[1] == -1 and idx[2] == -1
    if vm.hash_slot(vm.voxel(pts[3], 0.01), k) != vm.hash_slot(a, k):
        assert idx[3] == 1
    arr = m.arrays()
    np.testing.assert_array_equal(arr["means"][0], g["means"][0])
    np.testing.assert_array_equal(arr["f"][idx[idx >= 0]], g["f"][idx >= 0])


def test_sync_invariants():
    rng = np.random.default_rng(3)
    d = 4
    m = vm.GlobalMap(d=d, table_log2=16, voxel_size=0.05)
    m.insert(_gauss(rng, rng.uniform(-5, 5, size=(3000, 3)), d))
    local = {k: [] for k in vm.FIELDS}
    local["gidx"] = []
    for step, c in enumerate(([0, 0, 0], [1.0, 0.5, 0], [2.5, 1.0, 0.2], [-1, -1, 0])):
        c = np.array(c, np.float32)
        before = m.count
        if step:  # the local map learned something, and a few new Gaussians appeared
            local["f"] = [np.array(x, np.float32) + 1.0 for x in local["f"]]
            new = _gauss(rng, c + rng.uniform(-0.5, 0.5, size=(20, 3)), d)
            for k in vm.FIELDS:
                local[k] += [np.array(x, np.float32) for x in new[k]]
            local["gidx"] += [-1] * 20
        learned = {g: np.array(f) for g, f in zip(local["gidx"], local["f"]) if g >= 0}
        local = m.sync(local, c, 2.0)
        gidx = np.array(local["gidx"])
        assert m.count >= before
        assert len(set(gidx[gidx >= 0].tolist())) == int((gidx >= 0).sum())  # no duplicates
        assert np.all(vm.in_radius(np.array(local["means"]).reshape(-1, 3), c, 2.0))
        arr = m.arrays()
        near = set(np.flatnonzero(vm.in_radius(arr["means"], c, 2.0)).tolist())
        assert near <= set(gidx.tolist())  # every nearby global Gaussian is local
        for i, g in enumerate(gidx):
            if g >= 0:
                np.testing.assert_array_equal(arr["f"][g], local["f"][i])
        for g, f in learned.items():  # what the local map learned reached the global store
            np.testing.assert_array_equal(arr["f"][g], f)
