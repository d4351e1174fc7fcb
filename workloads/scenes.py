"""Seeded synthetic inputs for the per-keyframe latent-feature optimisation step.

This module only *draws* inputs: Gaussian primitives (Sec. III-A, Eq. gs_repr_basic
plus the query vector of Sec. III-B), a pinhole camera, a dictionary (keys/values)
and a target feature map with its validity mask.  It holds none of the method's
arithmetic (no projection, blending, decoding, loss or gradient), so the CPU oracle
and the CUDA path can both consume it without sharing any computation.

The paper's own workloads (TUM, Replica, FastCaMo RGB-D with CLIP/SAM targets,
Sec. IV-A) are not available; the scenes below stand in for them with the same
shapes and structure: d_s = 32 queries (Sec. III-B), D = 512-1024 dimensional
unit-norm targets that are piecewise constant over segments (mask-pooled VLM
embeddings, Sec. III-B), and 640x480 pinhole views of room-sized scenes.

All arrays are float32 / uint8, C-contiguous.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Camera:
    """Pinhole camera.  A world point p maps to camera space as R @ p + t;
    camera x points right, y down, z forward; pixel (x, y) has its centre at
    integer coordinates."""

    R: np.ndarray  # (3, 3) float32, world -> camera rotation (row-major)
    t: np.ndarray  # (3,) float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    z_near: float = 0.2

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


@dataclasses.dataclass
class Scene:
    name: str
    means: np.ndarray      # (N, 3)
    quats: np.ndarray      # (N, 4) (w, x, y, z), unit norm
    scales: np.ndarray     # (N, 3) linear scales
    opacities: np.ndarray  # (N,)
    f: np.ndarray          # (N, d) query vectors
    K: np.ndarray          # (M, d) dictionary keys
    V: np.ndarray          # (M, D) dictionary values (atoms)
    V0: np.ndarray         # (M, D) trust-region centre (initial dictionary)
    F: np.ndarray          # (H*W, D) target features, row = y*W + x
    mask: np.ndarray       # (H*W,) uint8, 1 = pixel in the loss set
    camera: Camera
    labels: np.ndarray | None = None  # (H*W,) int32 region id per pixel (-1 = none), for masks

    @property
    def n(self) -> int:
        return self.means.shape[0]

    @property
    def d(self) -> int:
        return self.f.shape[1]

    @property
    def M(self) -> int:
        return self.K.shape[0]

    @property
    def D(self) -> int:
        return self.V.shape[1]

    def crop(self, x0: int, y0: int, w: int, h: int, name: str | None = None) -> "Scene":
        """The (w, h) pixel window starting at (x0, y0) of this view, as its own
        camera (principal point shifted); Gaussians and dictionary are shared."""
        cam = self.camera
        assert 0 <= x0 and 0 <= y0 and x0 + w <= cam.width and y0 + h <= cam.height
        c2 = dataclasses.replace(cam, cx=cam.cx - x0, cy=cam.cy - y0, width=w, height=h)
        F = self.F.reshape(cam.height, cam.width, -1)[y0:y0 + h, x0:x0 + w].reshape(w * h, -1)
        m = self.mask.reshape(cam.height, cam.width)[y0:y0 + h, x0:x0 + w].reshape(-1)
        lab = None
        if self.labels is not None:
            lab = np.ascontiguousarray(self.labels.reshape(cam.height, cam.width)[y0:y0 + h, x0:x0 + w].reshape(-1))
        return dataclasses.replace(self, name=name or f"{self.name}[crop {x0},{y0} {w}x{h}]",
                                   camera=c2, F=np.ascontiguousarray(F), mask=np.ascontiguousarray(m), labels=lab)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _look_camera(position, forward, down, fx, fy, cx, cy, width, height, z_near=0.2) -> Camera:
    fwd = np.asarray(forward, np.float64)
    fwd /= np.linalg.norm(fwd)
    dn = np.asarray(down, np.float64)
    dn = dn - fwd * (dn @ fwd)
    dn /= np.linalg.norm(dn)
    right = np.cross(dn, fwd)  # x = y cross z for a right-handed (x right, y down, z fwd) frame
    R = np.stack([right, dn, fwd])
    t = -R @ np.asarray(position, np.float64)
    return Camera(R=_f32(R), t=_f32(t), fx=float(fx), fy=float(fy), cx=float(cx), cy=float(cy),
                  width=int(width), height=int(height), z_near=float(z_near))


def random_unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return _f32(q)


def _dictionary(rng, M, d, D):
    std = 1.0 / math.sqrt(d)
    K = _f32(rng.normal(0.0, std, size=(M, d)))
    V = _f32(rng.normal(0.0, std, size=(M, D)))
    return K, V


def _normalise_rows(x):
    return x / np.maximum(np.linalg.norm(x, axis=1, keepdims=True), 1e-12)


def tiny_scene(seed: int = 0, n: int = 2000, d: int = 16, M: int = 64, D: int = 512,
               width: int = 64, height: int = 48, fx: float = 60.0, mask_drop: float = 0.1) -> Scene:
    """The tiny plain-method case: Gaussians with means uniform in [-1,1]^3,
    log-normal scales (mu=-3, sigma=0.3), random unit quaternions, opacity
    U(0.1, 0.99), queries ~N(0,1); one pinhole camera at (0,0,-3) looking at the
    origin (up = -y).  Keys/values ~N(0, 1/sqrt(d)).  The target is a random sparse
    mixture (3 atoms, Dirichlet(1) weights) of a separate ground-truth dictionary
    per 8x8 pixel block, plus N(0, 0.01^2) noise, L2-normalised per pixel;
    a fraction `mask_drop` of the blocks is left out of the loss set."""
    rng = np.random.default_rng(seed)
    means = _f32(rng.uniform(-1.0, 1.0, size=(n, 3)))
    scales = _f32(np.exp(rng.normal(-3.0, 0.3, size=(n, 3))))
    quats = random_unit_quats(rng, n)
    opac = _f32(rng.uniform(0.1, 0.99, size=n))
    f = _f32(rng.normal(size=(n, d)))
    K, V = _dictionary(rng, M, d, D)
    cam = _look_camera((0, 0, -3), (0, 0, 1), (0, 1, 0), fx, fx, width / 2, height / 2, width, height)

    Vstar = rng.normal(size=(M, D))
    bw, bh = (width + 7) // 8, (height + 7) // 8
    F = np.zeros((height, width, D))
    mask = np.ones((height, width), np.uint8)
    for by in range(bh):
        for bx in range(bw):
            atoms = rng.choice(M, size=3, replace=False)
            w = rng.dirichlet(np.ones(3))
            mix = w @ Vstar[atoms]
            ys, xs = slice(by * 8, min(by * 8 + 8, height)), slice(bx * 8, min(bx * 8 + 8, width))
            blk = F[ys, xs]
            F[ys, xs] = mix[None, None, :] + rng.normal(0.0, 0.01, size=blk.shape)
            if rng.uniform() < mask_drop:
                mask[ys, xs] = 0
    F = _normalise_rows(F.reshape(-1, D))
    yy, xx = np.mgrid[0:height, 0:width]
    labels = ((yy // 8) * bw + xx // 8).astype(np.int32).reshape(-1)
    return Scene(name=f"tiny(seed={seed},N={n},{width}x{height},d={d},M={M},D={D})",
                 means=means, quats=quats, scales=scales, opacities=opac, f=f, K=K, V=V, V0=V.copy(),
                 F=_f32(F), mask=mask.reshape(-1), camera=cam, labels=labels)


# ----------------------------------------------------------------------------------------
# Room-shaped scenes
# ----------------------------------------------------------------------------------------

def _room_faces(rng, size, n_boxes):
    """Axis-aligned rectangles (origin, edge u, edge v, normal axis, object id, patch id)
    of a room of `size` (x, y, z; z up) and `n_boxes` random boxes standing on its floor."""
    Lx, Ly, Lz = size
    faces = []
    # room planes: (origin, u, v, normal axis); each split in two patches along u
    planes = [((0, 0, 0), (Lx, 0, 0), (0, Ly, 0), 2),    # floor
              ((0, 0, Lz), (Lx, 0, 0), (0, Ly, 0), 2),   # ceiling
              ((0, 0, 0), (0, Ly, 0), (0, 0, Lz), 0),    # wall x = 0
              ((Lx, 0, 0), (0, Ly, 0), (0, 0, Lz), 0),   # wall x = Lx
              ((0, 0, 0), (Lx, 0, 0), (0, 0, Lz), 1),    # wall y = 0
              ((0, Ly, 0), (Lx, 0, 0), (0, 0, Lz), 1)]   # wall y = Ly
    boxes = []
    for b in range(n_boxes):
        e = rng.uniform(0.2, 1.0, size=3)
        lo = np.array([rng.uniform(0.1, Lx - e[0] - 0.1), rng.uniform(0.1, Ly - e[1] - 0.1), 0.0])
        boxes.append((lo, lo + e))
        ex, ey, ez = e
        ox, oy, oz = lo
        # five faces (no bottom)
        faces += [((ox, oy, oz + ez), (ex, 0, 0), (0, ey, 0), 2, b),
                  ((ox, oy, oz), (0, ey, 0), (0, 0, ez), 0, b),
                  ((ox + ex, oy, oz), (0, ey, 0), (0, 0, ez), 0, b),
                  ((ox, oy, oz), (ex, 0, 0), (0, 0, ez), 1, b),
                  ((ox, oy + ey, oz), (ex, 0, 0), (0, 0, ez), 1, b)]
    for k, (o, u, v, ax) in enumerate(planes):
        u = np.asarray(u, float)
        for half in range(2):
            oo = np.asarray(o, float) + half * u / 2
            faces.append((tuple(oo), tuple(u / 2), v, ax, n_boxes + 2 * k + half))
    return faces, boxes


def _raycast_labels(cam: Camera, size, boxes, n_boxes):
    """Segment id of the first analytic surface hit by each pixel's ray (-1 if none)."""
    return _raycast(cam, size, boxes, n_boxes)[0]


def _raycast(cam: Camera, size, boxes, n_boxes):
    """Segment id and camera depth (0 if none) of the first surface hit by each pixel's ray."""
    H, W = cam.height, cam.width
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    dirc = np.stack([(xs - cam.cx) / cam.fx, (ys - cam.cy) / cam.fy, np.ones_like(xs)], -1).reshape(-1, 3)
    R = cam.R.astype(np.float64)
    dirw = dirc @ R  # R^T d
    origin = -R.T @ cam.t.astype(np.float64)
    n = dirw.shape[0]
    best_t = np.full(n, np.inf)
    label = np.full(n, -1, np.int64)
    Lx, Ly, Lz = size
    with np.errstate(divide="ignore", invalid="ignore"):
        # room interior planes
        plane_defs = [(2, 0.0, 0), (2, Lz, 1), (0, 0.0, 2), (0, Lx, 3), (1, 0.0, 4), (1, Ly, 5)]
        for ax, val, k in plane_defs:
            t = (val - origin[ax]) / dirw[:, ax]
            hit = origin[None, :] + t[:, None] * dirw
            ok = (t > 1e-9) & np.isfinite(t)
            for a2 in range(3):
                if a2 != ax:
                    ok &= (hit[:, a2] >= 0.0) & (hit[:, a2] <= size[a2])
            # patch split along the plane's first in-plane axis (u in _room_faces)
            uax = {2: 0, 0: 1, 1: 0}[ax]
            half = (hit[:, uax] > size[uax] / 2).astype(np.int64)
            upd = ok & (t < best_t)
            best_t[upd] = t[upd]
            label[upd] = n_boxes + 2 * k + half[upd]
        for b, (lo, hi) in enumerate(boxes):
            t0 = (lo[None, :] - origin[None, :]) / dirw
            t1 = (hi[None, :] - origin[None, :]) / dirw
            tmin = np.nanmax(np.minimum(t0, t1), axis=1)
            tmax = np.nanmin(np.maximum(t0, t1), axis=1)
            ok = (tmax >= tmin) & (tmin > 1e-9)
            upd = ok & (tmin < best_t)
            best_t[upd] = tmin[upd]
            label[upd] = b
    # the ray direction has camera-space z = 1, so the hit parameter is the camera depth
    depth = np.where(np.isfinite(best_t), best_t, 0.0)
    return label, depth


def room_scene(seed: int = 0, n: int = 300_000, d: int = 32, M: int = 256, D: int = 512,
               width: int = 640, height: int = 480, fx: float = 525.0, n_boxes: int = 20,
               size=(6.0, 5.0, 3.0), n_segments: int = 32, noise: float = 0.02) -> Scene:
    """Single room-shaped keyframe: N Gaussians on the 6 planes of a 6x5x3 m room and on
    20 random axis-aligned boxes (edges 0.2-1.0 m) standing on its floor, drawn in
    proportion to surface area.  Per-axis scales are log-normal around 1.5 cm (sigma 0.3)
    with the surface-normal axis x0.3, rotated by a random angle about the normal;
    opacity U(0.3, 0.99); queries ~N(0,1).  The camera stands in the room centre at
    1.5 m height with a seeded yaw, 640x480, fx = fy = 525.  Targets: each pixel's
    first-hit surface segment (boxes, plus each room plane split in two patches: 32
    segments) gets a random unit embedding, plus N(0, noise^2) per component,
    L2-normalised; the mask is the set of pixels that hit a surface."""
    rng = np.random.default_rng(seed)
    faces, boxes = _room_faces(rng, size, n_boxes)
    areas = np.array([np.linalg.norm(np.cross(u, v)) for (_, u, v, _, _) in faces])
    which = rng.choice(len(faces), size=n, p=areas / areas.sum())
    a = rng.uniform(size=n)
    b = rng.uniform(size=n)
    O = np.array([f[0] for f in faces], float)
    U = np.array([f[1] for f in faces], float)
    Vv = np.array([f[2] for f in faces], float)
    ax = np.array([f[3] for f in faces], int)
    means = O[which] + a[:, None] * U[which] + b[:, None] * Vv[which]
    scales = np.exp(rng.normal(math.log(0.015), 0.3, size=(n, 3)))
    nax = ax[which]
    scales[np.arange(n), nax] *= 0.3
    theta = rng.uniform(0, 2 * math.pi, size=n)
    quats = np.zeros((n, 4))
    quats[:, 0] = np.cos(theta / 2)
    quats[np.arange(n), 1 + nax] = np.sin(theta / 2)
    opac = rng.uniform(0.3, 0.99, size=n)
    f = rng.normal(size=(n, d))
    K, V = _dictionary(rng, M, d, D)
    yaw = rng.uniform(0, 2 * math.pi)
    centre = (size[0] / 2, size[1] / 2, 1.5)
    cam = _look_camera(centre, (math.cos(yaw), math.sin(yaw), 0.0), (0, 0, -1), fx, fx,
                       width / 2, height / 2, width, height)
    label = _raycast_labels(cam, size, boxes, n_boxes)
    n_ids = n_boxes + 12
    emb = _normalise_rows(rng.normal(size=(max(n_ids, n_segments), D)))
    F = emb[np.maximum(label, 0)] + rng.normal(0.0, noise, size=(label.shape[0], D))
    F = _normalise_rows(F)
    mask = (label >= 0).astype(np.uint8)
    F[mask == 0] = 0.0
    return Scene(name=f"room(seed={seed},N={n},{width}x{height},d={d},M={M},D={D})",
                 means=_f32(means), quats=_f32(quats), scales=_f32(scales), opacities=_f32(opac),
                 f=_f32(f), K=K, V=V, V0=V.copy(), F=_f32(F), mask=mask, camera=cam,
                 labels=label.astype(np.int32))


def room_rgbd(seed: int, scene: Scene, n_boxes: int = 20, size=(6.0, 5.0, 3.0), noise: float = 0.02):
    """Observed RGB-D of a room keyframe (the photometric and depth targets of the full Stage I
    objective): every surface segment a random colour, plus N(0, noise^2) per channel, clipped
    to [0, 1]; the ray-cast camera depth (0 where no surface is hit).  Also random initial
    Gaussian colours U(0, 1).  `seed` must be the seed the room was drawn with."""
    rng0 = np.random.default_rng(seed)
    _, boxes = _room_faces(rng0, size, n_boxes)
    label, depth = _raycast(scene.camera, size, boxes, n_boxes)
    rng = np.random.default_rng(seed + 3000)
    seg = rng.uniform(0.0, 1.0, size=(n_boxes + 12, 3))
    image = np.clip(seg[np.maximum(label, 0)] + rng.normal(0.0, noise, size=(label.shape[0], 3)), 0.0, 1.0)
    image[label < 0] = 0.0
    colours = rng.uniform(0.0, 1.0, size=(scene.n, 3))
    return _f32(colours), _f32(image), _f32(depth)


def room_views(seed: int = 0, n_views: int = 6, n: int = 300_000, d: int = 32, M: int = 256, D: int = 512,
               width: int = 640, height: int = 480, fx: float = 525.0, n_boxes: int = 20,
               size=(6.0, 5.0, 3.0), noise: float = 0.02) -> list:
    """Several keyframes of one room (the new keyframe plus sampled history keyframes): the
    Gaussians, queries and dictionary of room_scene(seed) seen from n_views cameras at the
    room centre with different seeded yaws and heights; each view has its own ray-cast target
    map (same segment embeddings).  The scenes share their Gaussian and dictionary arrays."""
    base = room_scene(seed, n=n, d=d, M=M, D=D, width=width, height=height, fx=fx, n_boxes=n_boxes, size=size,
                      noise=noise)
    rng = np.random.default_rng(seed + 1000)
    # rebuild the room's boxes and embeddings exactly as room_scene drew them
    rng0 = np.random.default_rng(seed)
    _, boxes = _room_faces(rng0, size, n_boxes)
    n_ids = n_boxes + 12
    emb_rng = np.random.default_rng(seed + 2000)
    emb = _normalise_rows(emb_rng.normal(size=(max(n_ids, 32), D)))
    views = []
    for v in range(n_views):
        if v == 0:
            cam = base.camera  # the new keyframe; its targets are redrawn with the shared embeddings
        else:
            yaw = rng.uniform(0, 2 * math.pi)
            h = rng.uniform(1.2, 1.8)
            centre = (size[0] / 2 + rng.uniform(-0.5, 0.5), size[1] / 2 + rng.uniform(-0.5, 0.5), h)
            cam = _look_camera(centre, (math.cos(yaw), math.sin(yaw), 0.0), (0, 0, -1), fx, fx, width / 2,
                               height / 2, width, height)
        label = _raycast_labels(cam, size, boxes, n_boxes)
        F = emb[np.maximum(label, 0)] + rng.normal(0.0, noise, size=(label.shape[0], D))
        F = _normalise_rows(F)
        mask = (label >= 0).astype(np.uint8)
        F[mask == 0] = 0.0
        views.append(dataclasses.replace(base, name=f"{base.name}[view {v}]", camera=cam, F=_f32(F), mask=mask,
                                         labels=label.astype(np.int32)))
    return views


def keyframe_batch(seed: int = 0, sizes=((320, 240), (640, 480), (848, 480)), ns=(100_000, 300_000, 200_000),
                   d: int = 32, M: int = 512, D: int = 768) -> list:
    """Keyframes of uneven resolution, each with its own room (independently seeded) and its own
    active map of Gaussians and queries, sharing one dictionary (the first room's K, V, V0):
    the shape of the batched workload (several keyframes, one dictionary).  Focal length
    scales with the image width (fx = 525 at 640)."""
    frames = []
    for k, ((w, h), n) in enumerate(zip(sizes, ns)):
        s = room_scene(seed + 97 * k, n=n, d=d, M=M, D=D, width=w, height=h, fx=525.0 * w / 640.0)
        frames.append(s)
    K, V, V0 = frames[0].K, frames[0].V, frames[0].V0
    return [dataclasses.replace(s, K=K, V=V, V0=V0, name=f"{s.name}[batch {k}]") for k, s in enumerate(frames)]


def precision_scene(seed: int = 0, **kw) -> Scene:
    """The larger-dims room: 500k Gaussians, d = 32, M = 512, D = 1024, 640x480."""
    args = dict(n=500_000, d=32, M=512, D=1024)
    args.update(kw)
    return room_scene(seed, **args)


def random_scene(seed: int, n: int, d: int, M: int, D: int, width: int, height: int,
                 fx: float | None = None, spread: float = 1.0, log_scale: float = -3.0,
                 opacity=(0.1, 0.99), depth: float = 3.0, mask_drop: float = 0.0) -> Scene:
    """A generic random scene for edge cases: means uniform in [-spread, spread]^3 in
    front of a camera at distance `depth`, random dictionary, random unit targets."""
    rng = np.random.default_rng(seed)
    means = _f32(rng.uniform(-spread, spread, size=(n, 3)))
    scales = _f32(np.exp(rng.normal(log_scale, 0.3, size=(n, 3))))
    quats = random_unit_quats(rng, n)
    opac = _f32(rng.uniform(opacity[0], opacity[1], size=n))
    f = _f32(rng.normal(size=(n, d)))
    K, V = _dictionary(rng, M, d, D)
    fx = fx if fx is not None else width * 0.94
    cam = _look_camera((0, 0, -depth), (0, 0, 1), (0, 1, 0), fx, fx, width / 2, height / 2, width, height)
    F = _normalise_rows(rng.normal(size=(width * height, D)))
    mask = (rng.uniform(size=width * height) >= mask_drop).astype(np.uint8)
    return Scene(name=f"random(seed={seed},N={n},{width}x{height},d={d},M={M},D={D})",
                 means=means, quats=quats, scales=scales, opacities=opac, f=f, K=K, V=V, V0=V.copy(),
                 F=_f32(F), mask=mask, camera=cam)


# ----------------------------------------------------------------------------------------
# Large map: a two-floor building
# ----------------------------------------------------------------------------------------

def building_gaussians(seed: int = 0, n: int = 2_000_000, d: int = 32, size=(20.0, 15.0, 6.0),
                       rooms=(4, 3), floors: int = 2) -> dict:
    """Gaussians of a 20 x 15 x 6 m building with two floors of 4 x 3 rooms: the floor and
    ceiling slab of every floor and the interior and exterior wall planes (each wall between
    rooms split by a 1 m door gap), sampled in proportion to surface area.  Per-axis log-normal
    scales around 1.5 cm (sigma 0.3), random unit quaternions, opacity U(0.3, 0.99), queries
    ~N(0, 1).  Returns the SoA arrays (float32) of the map."""
    rng = np.random.default_rng(seed)
    X, Y, Z = size
    fh = Z / floors
    quads = []  # (origin, edge u, edge v)
    for k in range(floors + 1):
        quads.append(((0.0, 0.0, k * fh), (X, 0.0, 0.0), (0.0, Y, 0.0)))
    for k in range(floors):
        z0 = k * fh
        for i in range(rooms[0] + 1):
            x = X * i / rooms[0]
            for j in range(rooms[1]):
                y0, y1 = Y * j / rooms[1], Y * (j + 1) / rooms[1]
                gap = 0 < i < rooms[0]
                mid = 0.5 * (y0 + y1)
                segs = [(y0, mid - 0.5), (mid + 0.5, y1)] if gap else [(y0, y1)]
                for a, b in segs:
                    quads.append(((x, a, z0), (0.0, b - a, 0.0), (0.0, 0.0, fh)))
        for j in range(rooms[1] + 1):
            y = Y * j / rooms[1]
            for i in range(rooms[0]):
                x0, x1 = X * i / rooms[0], X * (i + 1) / rooms[0]
                gap = 0 < j < rooms[1]
                mid = 0.5 * (x0 + x1)
                segs = [(x0, mid - 0.5), (mid + 0.5, x1)] if gap else [(x0, x1)]
                for a, b in segs:
                    quads.append(((a, y, z0), (b - a, 0.0, 0.0), (0.0, 0.0, fh)))
    O = np.array([q[0] for q in quads])
    U = np.array([q[1] for q in quads])
    V = np.array([q[2] for q in quads])
    area = np.linalg.norm(np.cross(U, V), axis=1)
    which = rng.choice(len(quads), size=n, p=area / area.sum())
    a, b = rng.uniform(size=n), rng.uniform(size=n)
    means = O[which] + a[:, None] * U[which] + b[:, None] * V[which]
    scales = np.exp(rng.normal(math.log(0.015), 0.3, size=(n, 3)))
    return dict(means=_f32(means), quats=random_unit_quats(rng, n), scales=_f32(scales),
                opacities=_f32(rng.uniform(0.3, 0.99, size=n)), f=_f32(rng.normal(size=(n, d))))
