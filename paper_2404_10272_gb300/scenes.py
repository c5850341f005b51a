"""Seeded synthetic inputs: occupancy grids, camera rays and blob fields.

This module only generates inputs.  It holds none of the sampler's
arithmetic (no step recurrence, no point location, no compositing), so the
CUDA path and the CPU oracle can both be fed from it without sharing any of
the method.

The paper's scenes (NeRF-Synthetic objects with one 128^3 grid, Mip-NeRF 360
unbounded scenes with four 128^3 cascade levels whose voxel size doubles per
level, Sec. 4.1) and its trained occupancy grids are not available, so these
generators reproduce their shapes: thin closed surfaces in a bounded box for
the object-centric case, and dense centre content with scattered clutter in
the outer cascade levels for the unbounded case.

Conventions shared by every generator:
  * occupancy grids are uint8 [L, R, R, R], C order, x slowest, level 0
    finest; level boxes are half-open [lo, hi) given as float32 [L, 6]
    (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z);
  * rays are float32 [N, 3] origins and unit directions, normalised in
    float64 and then rounded; pixel (px, py) is ray py * W + px, pixel
    centres at +0.5, horizontal field of view, z up;
  * a Gaussian-blob field is float32 [G, 8]: mu_x, mu_y, mu_z, s, a, r, g, b.
"""
from __future__ import annotations

import copy
from dataclasses import dataclass, field as dc_field
import functools
import math

import numpy as np

__all__ = [
    "Scene", "Camera", "SamplerParams", "random_rotation", "ellipsoid_occupancy",
    "dilate", "box_occupancy", "cascade_boxes", "look_at_rays", "orbit_camera",
    "gaussian_field", "tiny_scene", "object_scene", "unbounded_scene",
    "object_cameras", "tiny_camera", "unbounded_camera", "random_grid", "cascade_from",
    "batch_jobs",
]


@dataclass
class SamplerParams:
    near: float
    far: float
    step: float
    cone: float = 0.0
    max_step: float = 1e10
    max_steps: int = 1 << 20


@dataclass
class Scene:
    occ: np.ndarray            # uint8 [L, R, R, R]
    aabbs: np.ndarray          # float32 [L, 6]
    params: SamplerParams
    field: np.ndarray | None = None   # float32 [G, 8]
    name: str = ""
    info: dict = dc_field(default_factory=dict)

    @property
    def levels(self) -> int:
        return int(self.occ.shape[0])

    @property
    def res(self) -> int:
        return int(self.occ.shape[1])


@dataclass
class Camera:
    eye: np.ndarray
    target: np.ndarray
    width: int
    height: int
    fov: float
    up: np.ndarray = dc_field(default_factory=lambda: np.array([0.0, 0.0, 1.0]))

    def rays(self):
        return look_at_rays(self.eye, self.target, self.width, self.height, self.fov, self.up)


# ---------------------------------------------------------------------------
# occupancy
# ---------------------------------------------------------------------------

def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix (QR of a Gaussian matrix, sign-fixed)."""
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _voxel_centres(R: int, lo, hi) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    axes = [lo[c] + (np.arange(R) + 0.5) * (hi[c] - lo[c]) / R for c in range(3)]
    return np.meshgrid(*axes, indexing="ij")


def ellipsoid_occupancy(R, lo, hi, centres, semi_axes, rotations, thickness=None,
                        solid=False) -> np.ndarray:
    """uint8 [R, R, R]: voxels whose centre lies within `thickness` of an
    ellipsoid surface (approximate distance |‖q‖ - 1| * min(axes), q the
    point in the ellipsoid's unit frame), or inside it when `solid`."""
    X, Y, Z = _voxel_centres(R, lo, hi)
    P = np.stack([X, Y, Z], -1)
    out = np.zeros((R, R, R), bool)
    for c, ax, rot in zip(centres, semi_axes, rotations):
        q = ((P - c) @ rot) / ax
        rho = np.linalg.norm(q, axis=-1)
        if solid:
            out |= rho <= 1.0
        else:
            out |= np.abs(rho - 1.0) * np.min(ax) <= thickness
    return out.astype(np.uint8)


def dilate(occ: np.ndarray, r: int = 1) -> np.ndarray:
    """(2r+1)^3 binary dilation with zero padding."""
    a = occ.astype(bool)
    out = a.copy()
    R = a.shape
    for dx in range(-r, r + 1):
        for dy in range(-r, r + 1):
            for dz in range(-r, r + 1):
                src = a[max(0, -dx):R[0] - max(0, dx), max(0, -dy):R[1] - max(0, dy),
                        max(0, -dz):R[2] - max(0, dz)]
                out[max(0, dx):R[0] - max(0, -dx), max(0, dy):R[1] - max(0, -dy),
                    max(0, dz):R[2] - max(0, -dz)] |= src
    return out.astype(np.uint8)


def box_occupancy(R, lo, hi, boxes) -> np.ndarray:
    """uint8 [R, R, R]: voxels whose centre lies in any (bmin, bmax) box."""
    X, Y, Z = _voxel_centres(R, lo, hi)
    out = np.zeros((R, R, R), bool)
    for bmin, bmax in boxes:
        out |= ((X >= bmin[0]) & (X < bmax[0]) & (Y >= bmin[1]) & (Y < bmax[1])
                & (Z >= bmin[2]) & (Z < bmax[2]))
    return out.astype(np.uint8)


def cascade_boxes(levels: int, half: float = 1.0) -> np.ndarray:
    """Level l box = [-half*2^l, half*2^l)^3 (voxel size doubles per level)."""
    out = np.zeros((levels, 6), np.float32)
    for l in range(levels):
        h = half * (2.0 ** l)
        out[l] = [-h, -h, -h, h, h, h]
    return out


def random_grid(rng: np.random.Generator, levels: int, res: int, p: float) -> np.ndarray:
    """Independent Bernoulli(p) voxels, uint8 [L, R, R, R] (property tests)."""
    return (rng.random((levels, res, res, res)) < p).astype(np.uint8)


# ---------------------------------------------------------------------------
# cameras
# ---------------------------------------------------------------------------

def look_at_rays(eye, target, W: int, H: int, fov: float, up=(0.0, 0.0, 1.0)):
    """Pinhole rays: float32 origins [W*H, 3] and unit directions [W*H, 3]."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.asarray(up, np.float64)
    if abs(np.dot(f, up)) > 0.999:
        up = np.array([0.0, 1.0, 0.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(0.5 * fov)
    px = (np.arange(W) + 0.5) / W * 2.0 - 1.0
    py = 1.0 - (np.arange(H) + 0.5) / H * 2.0
    U, V = np.meshgrid(px * th, py * th * (H / W), indexing="xy")
    d = f[None, None, :] + U[..., None] * r + V[..., None] * u
    d = d.reshape(-1, 3)
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    o = np.broadcast_to(eye, d.shape)
    return np.ascontiguousarray(o, np.float32), np.ascontiguousarray(d, np.float32)


def orbit_camera(rng: np.random.Generator, radius: float, W: int, H: int, fov: float,
                 upper: bool = True) -> Camera:
    az = rng.uniform(0.0, 2.0 * math.pi)
    el = rng.uniform(0.1, 1.2) if upper else rng.uniform(-1.2, 1.2)
    eye = radius * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    return Camera(eye=eye, target=np.zeros(3), width=W, height=H, fov=fov)


# ---------------------------------------------------------------------------
# blob field (stand-in for the trained radiance field)
# ---------------------------------------------------------------------------

def gaussian_field(rng: np.random.Generator, n: int = 64, shell: float = 0.9,
                   spread: float = 0.35) -> np.ndarray:
    """float32 [n, 8]: blob centres near a random shell, s ~ U[0.03, 0.15],
    a ~ U[5, 50], rgb ~ U[0, 1]^3."""
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=-1, keepdims=True)
    rad = shell + rng.uniform(-spread, spread, size=(n, 1))
    out = np.zeros((n, 8), np.float32)
    out[:, 0:3] = dirs * rad
    out[:, 3] = rng.uniform(0.03, 0.15, size=n)
    out[:, 4] = rng.uniform(5.0, 50.0, size=n)
    out[:, 5:8] = rng.uniform(0.0, 1.0, size=(n, 3))
    return out


# ---------------------------------------------------------------------------
# the three workload shapes
# ---------------------------------------------------------------------------

def _shells(rng, n, c_range, a_range):
    centres = rng.uniform(-c_range, c_range, size=(n, 3))
    axes = rng.uniform(a_range[0], a_range[1], size=(n, 3))
    rots = [random_rotation(rng) for _ in range(n)]
    return centres, axes, rots


def _cached_scene(fn):
    """Scenes take seconds to generate; keep one per argument set and hand out copies."""
    cached = functools.lru_cache(maxsize=8)(fn)

    @functools.wraps(fn)
    def wrapper(*args, **kwargs):
        return copy.deepcopy(cached(*args, **kwargs))
    return wrapper


@_cached_scene
def tiny_scene(seed: int = 1001) -> Scene:
    """One 64^3 level over [-1.5, 1.5)^3; shells of 3 random ellipsoids
    (voxel centres within 0.05 of a surface); near 2, far 6, step 5e-3."""
    rng = np.random.default_rng(seed)
    R, lo, hi = 64, [-1.5] * 3, [1.5] * 3
    c, a, rot = _shells(rng, 3, 0.8, (0.3, 0.9))
    occ = ellipsoid_occupancy(R, lo, hi, c, a, rot, thickness=0.05)[None]
    aabbs = np.array([lo + hi], np.float32)
    p = SamplerParams(near=2.0, far=6.0, step=5e-3, cone=0.0)
    return Scene(occ=occ, aabbs=aabbs, params=p, field=gaussian_field(rng), name="tiny-64^3",
                 info={"occupancy": float(occ.mean())})


def tiny_camera(seed: int = 1001) -> Camera:
    return orbit_camera(np.random.default_rng(seed + 1), 4.0, 96, 96, 0.69)


@_cached_scene
def object_scene(seed: int = 1002, R: int = 128) -> Scene:
    """One 128^3 level over [-1.5, 1.5)^3: 8 thin ellipsoidal shells plus 2
    solid ellipsoids, dilated by one voxel; near 2, far 6,
    step = fl32(sqrt(3) * 3 / 1024); 64-blob field."""
    rng = np.random.default_rng(seed)
    lo, hi = [-1.5] * 3, [1.5] * 3
    c, a, rot = _shells(rng, 8, 0.6, (0.25, 0.8))
    occ = ellipsoid_occupancy(R, lo, hi, c, a, rot, thickness=0.006)
    c2, a2, rot2 = _shells(rng, 2, 0.5, (0.1, 0.25))
    occ |= ellipsoid_occupancy(R, lo, hi, c2, a2, rot2, solid=True)
    occ = dilate(occ, 1)[None]
    aabbs = np.array([lo + hi], np.float32)
    step = float(np.float32(math.sqrt(3.0) * 3.0 / 1024.0))
    p = SamplerParams(near=2.0, far=6.0, step=step, cone=0.0)
    return Scene(occ=occ, aabbs=aabbs, params=p, field=gaussian_field(rng), name="object-128^3",
                 info={"occupancy": float(occ.mean())})


def object_cameras(seed: int = 1002, n: int = 20, W: int = 800, H: int = 800) -> list[Camera]:
    return [orbit_camera(np.random.default_rng(seed + 1 + j), 4.0, W, H, 0.69) for j in range(n)]


@_cached_scene
def unbounded_scene(seed: int = 1003, levels: int = 4, R: int = 128) -> Scene:
    """Four 128^3 cascade levels, level l over [-2^l, 2^l)^3: ellipsoidal
    shells at the centre of level 0 and random axis-aligned boxes in the
    outer shell region of every coarser level; near 0.02, far 1e3,
    step 1.73e-3, cone 0.004 (linearly growing step)."""
    rng = np.random.default_rng(seed)
    aabbs = cascade_boxes(levels, 1.0)
    occ = np.zeros((levels, R, R, R), np.uint8)
    lo0, hi0 = aabbs[0, :3], aabbs[0, 3:]
    c, a, rot = _shells(rng, 6, 0.4, (0.2, 0.6))
    occ[0] = dilate(ellipsoid_occupancy(R, lo0, hi0, c, a, rot, thickness=0.008), 1)
    for l in range(1, levels):
        h, hin = 2.0 ** l, 2.0 ** (l - 1)
        nb = int(rng.integers(20, 201))
        boxes = []
        while len(boxes) < nb:
            ctr = rng.uniform(-h, h, size=3)
            if np.all(np.abs(ctr) < hin):
                continue   # keep clutter in the shell region of this level
            ext = rng.uniform(0.02, 0.12, size=3) * h
            boxes.append((ctr - ext, ctr + ext))
        occ[l] = box_occupancy(R, aabbs[l, :3], aabbs[l, 3:], boxes)
    p = SamplerParams(near=0.02, far=1e3, step=1.73e-3, cone=0.004, max_step=1e10)
    info = {"occupancy_per_level": [float(occ[l].mean()) for l in range(levels)]}
    return Scene(occ=occ, aabbs=aabbs, params=p, field=gaussian_field(rng), name="unbounded-4x128^3",
                 info=info)


def unbounded_camera(seed: int = 1003, W: int = 1245, H: int = 825, j: int = 0) -> Camera:
    rng = np.random.default_rng(seed + 1 + j)
    eye = rng.uniform(-0.5, 0.5, size=3)
    dirn = rng.normal(size=3)
    dirn /= np.linalg.norm(dirn)
    return Camera(eye=eye, target=eye + dirn, width=W, height=H, fov=1.0)


# ---------------------------------------------------------------------------
# batching workload: many (scene, camera) jobs
# ---------------------------------------------------------------------------

def cascade_from(base: np.ndarray, levels: int, rng: np.random.Generator, half: float = 1.5):
    """A cascade whose level 0 is `base` (R^3 over [-half, half)^3) and whose level l covers
    [-half*2^l, half*2^l)^3: its central half holds the 2x OR-pooled level l-1 (as a trained
    cascade would) and its outer shell a few random boxes."""
    R = base.shape[0]
    occ = np.zeros((levels, R, R, R), np.uint8)
    occ[0] = base
    aabbs = cascade_boxes(levels, half)
    for l in range(1, levels):
        pooled = occ[l - 1].reshape(R // 2, 2, R // 2, 2, R // 2, 2).max(axis=(1, 3, 5))
        q = R // 4
        occ[l, q:q + R // 2, q:q + R // 2, q:q + R // 2] = pooled
        h, hin = aabbs[l, 3], aabbs[l - 1, 3]
        boxes = []
        while len(boxes) < 12:
            ctr = rng.uniform(-h, h, size=3)
            if np.all(np.abs(ctr) < hin):
                continue
            ext = rng.uniform(0.03, 0.1, size=3) * h
            boxes.append((ctr - ext, ctr + ext))
        occ[l] |= box_occupancy(R, aabbs[l, :3], aabbs[l, 3:], boxes)
    return occ, aabbs


def batch_jobs(seed: int = 1004, n: int = 64, min_side: int = 64, max_side: int = 800):
    """`n` jobs drawn from the tiny-type and object-type scenes: kind, cascade depth 1..4,
    image width and height uniform in [min_side, max_side], a camera on the radius-4 upper
    hemisphere.  Returns (scenes, jobs): scenes[(kind, levels)] = Scene, and per job a dict
    with scene key, width, height and rays."""
    rng = np.random.default_rng(seed)
    scenes_out = {}
    jobs = []
    for j in range(n):
        kind = "tiny" if rng.random() < 0.5 else "object"
        levels = int(rng.integers(1, 5))
        W = int(rng.integers(min_side, max_side + 1))
        H = int(rng.integers(min_side, max_side + 1))
        key = (kind, levels)
        if key not in scenes_out:
            base = tiny_scene() if kind == "tiny" else object_scene()
            occ, aabbs = cascade_from(base.occ[0], levels, np.random.default_rng(seed * 10 + levels))
            scenes_out[key] = Scene(occ=occ, aabbs=aabbs, params=base.params, field=base.field,
                                    name=f"{kind}-L{levels}")
        cam = orbit_camera(rng, 4.0, W, H, 0.69)
        o, d = cam.rays()
        jobs.append({"scene": key, "width": W, "height": H, "rays_o": o, "rays_d": d})
    return scenes_out, jobs
