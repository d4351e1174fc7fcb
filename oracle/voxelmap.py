"""Oracle of the voxel-hashed local/global map management (Sec. III-E, "Local-Global Map
Management via Voxel Hashing").

TEST INFRASTRUCTURE ONLY (imported by tests/ and never by the product path).

Plain Python, one Gaussian at a time in input order, integers and float32 decisions taken with
the same roundings as the definition below, so the GPU map must match it bit for bit.

Readings, where the paper is silent:
  * voxel v = floor(p / s_v) per axis, p / s_v evaluated in float32 (s_v = 0.01 m by default);
  * the hash of a voxel is the spatial hash of Teschner et al. (2003): the xor of the three
    coordinates times the primes 73856093, 19349663, 83492791, on 64-bit two's-complement
    integers, reduced modulo the table size T = 2^k (its low k bits).  The table stores no
    key: two voxels with the same slot collide, and the second one is treated as occupied
    (the paper accepts such collisions as rare and harmless);
  * insert-if-free: in input order, a Gaussian whose slot is empty takes the next free index
    of the global store and the slot; one whose slot is taken is not inserted;
  * the active set of a camera position c and radius r: the Gaussians with
    (dx*dx + dy*dy) + dz*dz <= r*r, dx = x - c_x ..., every operation rounded to float32;
  * synchronisation (the paper's two steps): Local -> Global first, so that nothing a local
    Gaussian learned is lost when it leaves the active set: a local Gaussian that came from the
    global store (global index >= 0) overwrites its entry; a new one (index -1) is inserted if
    its slot is free.  Then Global -> Local: the local Gaussians outside the radius are dropped
    (the rest keep their order), and the global Gaussians inside the radius that are not in the
    local map are appended in global-index order.  A Gaussian keeps the slot of the voxel it
    was inserted from (the key is not recomputed when it moves).

Parity status: pinned by tests/test_oracle_voxelmap.py (hand-computed hashes and voxels on cell
boundaries, brute-force radius filters, insert order and collisions on hand-built cases, the
invariants of a synchronisation sequence).
"""
from __future__ import annotations

import numpy as np

PRIMES = (73856093, 19349663, 83492791)
FIELDS = ("means", "quats", "scales", "opacities", "f")


def voxel(p, s_v: float) -> np.ndarray:
    """floor(p / s_v) per axis with the division rounded to float32 (int64 result)."""
    q = np.asarray(p, np.float32) / np.float32(s_v)
    return np.floor(q).astype(np.int64)


def _wrap64(x: int) -> int:
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >= 1 << 63 else x


def hash_slot(v, table_log2: int) -> int:
    """Slot of voxel v = (x, y, z): (x p1 ^ y p2 ^ z p3) mod 2^table_log2 on 64-bit integers."""
    x, y, z = (int(c) for c in v)
    h = _wrap64(_wrap64(x * PRIMES[0]) ^ _wrap64(y * PRIMES[1]) ^ _wrap64(z * PRIMES[2]))
    return h & ((1 << table_log2) - 1)


def in_radius(means, c, r: float) -> np.ndarray:
    """(dx*dx + dy*dy) + dz*dz <= r*r in float32, operation by operation."""
    m = np.asarray(means, np.float32)
    c = np.asarray(c, np.float32)
    d = m - c[None, :]
    s = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    return s <= np.float32(r) * np.float32(r)


class GlobalMap:
    """The global store (attribute rows in index order) and the slot table (-1 = empty)."""

    def __init__(self, d: int, table_log2: int, voxel_size: float = 0.01):
        self.d, self.table_log2, self.voxel_size = d, table_log2, voxel_size
        self.table = np.full(1 << table_log2, -1, np.int64)
        self.rows = {k: [] for k in FIELDS}

    @property
    def count(self) -> int:
        return len(self.rows["means"])

    def arrays(self) -> dict:
        shapes = dict(means=3, quats=4, scales=3, opacities=1, f=self.d)
        out = {}
        for k in FIELDS:
            a = np.asarray(self.rows[k], np.float32).reshape(self.count, shapes[k])
            out[k] = a[:, 0] if k == "opacities" else a
        return out

    def slot_of(self, p) -> int:
        return hash_slot(voxel(p, self.voxel_size), self.table_log2)

    def insert(self, g: dict) -> np.ndarray:
        """Insert-if-free of the rows of g in order; returns each row's global index or -1."""
        n = len(g["means"])
        out = np.full(n, -1, np.int64)
        for i in range(n):
            s = self.slot_of(g["means"][i])
            if self.table[s] >= 0:
                continue
            idx = self.count
            self.table[s] = idx
            for k in FIELDS:
                self.rows[k].append(np.array(g[k][i], np.float32))
            out[i] = idx
        return out

    def write_back(self, local: dict) -> np.ndarray:
        """Local -> Global: entries of known Gaussians overwritten, new ones inserted if free.
        Returns the (possibly new) global index of every local row."""
        gidx = np.array(local["gidx"], np.int64)
        for i in range(len(gidx)):
            if gidx[i] >= 0:
                for k in FIELDS:
                    self.rows[k][gidx[i]] = np.array(local[k][i], np.float32)
        new = np.flatnonzero(gidx < 0)
        if new.size:
            got = self.insert({k: [local[k][i] for i in new] for k in FIELDS})
            gidx[new] = got
        return gidx

    def sync(self, local: dict, c, r: float) -> dict:
        """Local -> Global, then Global -> Local around c with radius r; returns the new local
        map (rows in order: the kept local rows, then the appended global rows)."""
        gidx = self.write_back(local)
        keep = in_radius(local["means"], c, r) if len(gidx) else np.zeros(0, bool)
        # a new local Gaussian that found its slot taken has no global entry: it stays local
        # only while inside the radius, like the others
        out = {k: [np.array(local[k][i], np.float32) for i in np.flatnonzero(keep)] for k in FIELDS}
        out["gidx"] = [int(gidx[i]) for i in np.flatnonzero(keep)]
        present = {g for g in out["gidx"] if g >= 0}
        arr = self.arrays()
        near = np.flatnonzero(in_radius(arr["means"], c, r)) if self.count else np.zeros(0, np.int64)
        for g in near:
            if int(g) in present:
                continue
            for k in FIELDS:
                out[k].append(np.array(arr[k][g], np.float32))
            out["gidx"].append(int(g))
        return out
