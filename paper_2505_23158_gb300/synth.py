"""Seeded synthetic inputs: scenes, chunk centres, depth thresholds and cameras.

This module is shared by the CUDA path's callers (tests, bench, smoke) and by
the oracle's callers.  It draws raw Gaussian parameters and camera poses and
nothing else: no activation, projection, selection or blending arithmetic of
the method lives here.  Every array is produced by numpy's PCG64 generator
seeded with an explicit (seed, stream) tuple, so both sides see identical
bytes.

Workloads (sizes follow the paper's large outdoor/indoor captures, Sec. 4 and
the supplementary "Datasets" section; the paper's datasets are not available,
so these synthetic scenes stand in for them):

* ``plain_scene``      - single-level scene of N Gaussians in [-1,1]^3
                         (4,096 by default) viewed by ``plain_camera``.
* ``outdoor_scene``    - heightfield world with L LOD levels (level l holds
                         N0 / 4^l Gaussians, scales doubling per level), a
                         regular chunk grid and a camera trajectory.
* ``finetune_scene``   - one chunk cell of the outdoor generator.
* ``ray_scene``        - tiny Gaussians at given distances on tile-centre rays
                         (one tile key each), for counting checks.
* ``large_scene``      - 80M Gaussians over 6 levels: the outdoor heightfield
                         with room-like indoor blocks (walls, floors) on a
                         quarter of the chunk cells, 32x32 chunks, viewed by
                         batches of 3840x2160 street cameras.

Raw parameter layout (host, float32, C-contiguous), per level:
  means           (N, 3)   world position, metres (outdoor) or units (plain)
  log_scales      (N, 3)   natural log of the per-axis standard deviation
  quats           (N, 4)   (w, x, y, z), not normalised
  opacity_logits  (N,)     logit of the opacity
  sh              (N, 16, 3)  degree-3 SH coefficients, coefficient-major,
                              channel-minor, real basis order l, m=-l..l
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

SH_COEFFS = 16


# --------------------------------------------------------------------------
# containers
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Level:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    filter_var: float = 0.0  # variance of the per-level 3D smoothing filter

    @property
    def n(self) -> int:
        return int(self.means.shape[0])


@dataclasses.dataclass
class Scene:
    levels: List[Level]
    d_thresholds: np.ndarray            # (L-1,) float64, metres, ascending
    chunk_centers: np.ndarray           # (K, 3) float64
    sh_degree: int = 3
    extent: float = 0.0                 # side of the square world (outdoor)
    height_params: Optional[dict] = None
    filter2d: bool = False              # opacity-compensated 2D filter (Mip-Splatting)

    @property
    def num_levels(self) -> int:
        return len(self.levels)

    @property
    def n_total(self) -> int:
        return sum(l.n for l in self.levels)


@dataclasses.dataclass
class Camera:
    """Pinhole camera, world->camera p_c = R p_w + t, OpenCV axes
    (x right, y down, z forward).  ``center`` is the camera position in
    world coordinates, in float64."""
    R: np.ndarray          # (3, 3) float32
    t: np.ndarray          # (3,) float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float
    center: np.ndarray     # (3,) float64


# --------------------------------------------------------------------------
# camera construction (look-at)
# --------------------------------------------------------------------------
def look_at(position, forward, up, width, height, fov_y_deg, znear=0.2) -> Camera:
    """Camera at ``position`` looking along ``forward`` with world ``up``.
    fov_y is the vertical field of view; fx = fy = (H/2)/tan(fov_y/2),
    principal point at the image centre."""
    p = np.asarray(position, dtype=np.float64)
    f = np.asarray(forward, dtype=np.float64)
    f = f / np.linalg.norm(f)
    u = np.asarray(up, dtype=np.float64)
    x = np.cross(f, u)
    x = x / np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f]).astype(np.float64)
    t = -R @ p
    foc = (height / 2.0) / math.tan(math.radians(fov_y_deg) / 2.0)
    return Camera(R=R.astype(np.float32), t=t.astype(np.float32),
                  fx=float(np.float32(foc)), fy=float(np.float32(foc)),
                  cx=width / 2.0, cy=height / 2.0, width=int(width),
                  height=int(height), znear=float(znear), center=p.copy())


# --------------------------------------------------------------------------
# plain single-level scene (CPU-oracle sized)
# --------------------------------------------------------------------------
def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), *[int(s) for s in stream]])


def plain_scene(seed: int = 0, n: int = 4096, log_scale_mean: float = -3.5,
                log_scale_std: float = 0.5, sh_std: float = 0.2) -> Scene:
    """N Gaussians: means U[-1,1]^3, log-scales N(-3.5, 0.5) per axis,
    quaternions N(0, I4) (uniform rotation once normalised), opacity logit
    N(0, 1), all 48 SH coefficients N(0, 0.2).  One level, no chunks."""
    r = _rng(seed, 0)
    means = r.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    log_scales = r.normal(log_scale_mean, log_scale_std, size=(n, 3)).astype(np.float32)
    quats = r.normal(0.0, 1.0, size=(n, 4)).astype(np.float32)
    logits = r.normal(0.0, 1.0, size=(n,)).astype(np.float32)
    sh = r.normal(0.0, sh_std, size=(n, SH_COEFFS, 3)).astype(np.float32)
    lvl = Level(means, log_scales, quats, logits, sh, 0.0)
    return Scene(levels=[lvl], d_thresholds=np.zeros(0, np.float64),
                 chunk_centers=np.zeros((1, 3), np.float64), sh_degree=3)


def plain_camera(width: int = 256, height: int = 256, fov_y_deg: float = 60.0) -> Camera:
    """Camera at (0,0,-3) looking at the origin, image y axis along world +y
    (world up is -y), so R = I and t = (0, 0, 3)."""
    return look_at((0.0, 0.0, -3.0), (0.0, 0.0, 1.0), (0.0, -1.0, 0.0),
                   width, height, fov_y_deg)


def ray_scene(level_distances: Sequence[Sequence[float]], width: int = 256, height: int = 256,
              fov_y_deg: float = 60.0):
    """Scene whose every Gaussian yields exactly one tile key: level l holds
    one tiny, nearly opaque Gaussian per entry of ``level_distances[l]``,
    placed at that distance (metres) from the camera centre on the ray
    through the centre of a 16x16 tile (tiles taken in turn).  The camera
    sits at the origin looking along +z (R = I, t = 0).  Returns (scene,
    camera); the tile-key count of any active set is then the number of its
    Gaussians."""
    cam = look_at((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), (0.0, -1.0, 0.0), width, height, fov_y_deg)
    tx, ty = width // 16, height // 16
    levels = []
    slot = 0
    for dl in level_distances:
        dl = np.asarray(dl, np.float64)
        means = np.zeros((dl.size, 3))
        for i, dist in enumerate(dl):
            t = slot % (tx * ty)
            slot += 1
            u = 16.0 * (t % tx) + 8.0
            v = 16.0 * (t // tx) + 8.0
            ray = np.array([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, 1.0])
            means[i] = dist * ray / np.linalg.norm(ray)
        n = dl.size
        levels.append(Level(means=means.astype(np.float32),
                            log_scales=np.full((n, 3), -12.0, np.float32),
                            quats=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                            opacity_logits=np.full(n, 5.0, np.float32),
                            sh=np.zeros((n, SH_COEFFS, 3), np.float32)))
    L = len(levels)
    scene = Scene(levels=levels, d_thresholds=np.array([10.0 * 2 ** l for l in range(L - 1)]),
                  chunk_centers=np.zeros((1, 3)))
    return scene, cam


# --------------------------------------------------------------------------
# outdoor heightfield world
# --------------------------------------------------------------------------
def height_params(seed: int, amplitude: float = 20.0, octaves: int = 4) -> dict:
    """Sum of ``octaves`` sinusoids: a_k proportional to 2^-k with
    sum a_k = amplitude, f_k = 2^k * 2 cycles per km, seeded direction and
    phase."""
    r = _rng(seed, 100)
    a = np.array([2.0 ** -k for k in range(octaves)])
    a = a * (amplitude / a.sum())
    f = np.array([2.0 ** k * 2.0 for k in range(octaves)])
    theta = r.uniform(0, 2 * math.pi, size=octaves)
    phi = r.uniform(0, 2 * math.pi, size=octaves)
    return dict(a=a, f=f, theta=theta, phi=phi)


def height(hp: dict, x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    h = np.zeros(np.broadcast(x, y).shape, dtype=np.float64)
    for a, f, th, ph in zip(hp["a"], hp["f"], hp["theta"], hp["phi"]):
        h += a * np.sin(2 * math.pi * f * (x * math.cos(th) + y * math.sin(th)) / 1000.0 + ph)
    return h


def _morton_order(x: np.ndarray, y: np.ndarray, extent: float) -> np.ndarray:
    """Stable permutation putting points in Z-order of a 2^16 x 2^16 grid.
    Trained scenes exported per region have this kind of spatial coherence;
    it is an input property, the library does not rely on it for
    correctness."""
    qx = np.clip((x / max(extent, 1e-9) * 65535.0), 0, 65535).astype(np.uint64)
    qy = np.clip((y / max(extent, 1e-9) * 65535.0), 0, 65535).astype(np.uint64)

    def spread(v):
        v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF)
        v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F)
        v = (v | (v << np.uint64(2))) & np.uint64(0x33333333)
        v = (v | (v << np.uint64(1))) & np.uint64(0x55555555)
        return v

    code = spread(qx) | (spread(qy) << np.uint64(1))
    return np.argsort(code, kind="stable")


def outdoor_scene(seed: int = 0, n0: int = 16_000_000, num_levels: int = 4,
                  extent: float = 1000.0, grid: int = 16,
                  d_thresholds: Sequence[float] = (10.0, 20.0, 40.0),
                  log_scale_mean0: float = math.log(0.125),
                  jitter0: float = 0.5, sh_std: float = 0.2,
                  cam_height: float = 2.0, spatial_order: bool = True,
                  filter_vars: Optional[Sequence[float]] = None,
                  region: Optional[Sequence[float]] = None) -> Scene:
    """Outdoor LOD scene on a seeded heightfield over [0, extent]^2 (z up).

    Level l has n0 / 4^l Gaussians at uniform (x, y) (inside ``region`` =
    (x0, y0, x1, y1) when given), placed on the heightfield and jittered
    N(0, (jitter0 * 2^l)^2) per axis; log-scales N(log_scale_mean0 + l ln 2,
    0.5); opacity logit N(1, 1); SH N(0, sh_std).  Chunk centres are the
    centres of a ``grid`` x ``grid`` partition, at cam_height above ground.
    """
    hp = height_params(seed)
    levels = []
    x0, y0, x1, y1 = region if region is not None else (0.0, 0.0, extent, extent)
    for l in range(num_levels):
        n = max(int(n0 // (4 ** l)), 1)
        r = _rng(seed, 1, l)
        xy = np.empty((n, 2), np.float64)
        xy[:, 0] = r.uniform(x0, x1, size=n)
        xy[:, 1] = r.uniform(y0, y1, size=n)
        z = height(hp, xy[:, 0], xy[:, 1])
        jit = r.normal(0.0, jitter0 * 2.0 ** l, size=(n, 3))
        means = np.empty((n, 3), np.float32)
        means[:, 0] = xy[:, 0] + jit[:, 0]
        means[:, 1] = xy[:, 1] + jit[:, 1]
        means[:, 2] = z + jit[:, 2]
        del xy, z, jit
        log_scales = r.normal(log_scale_mean0 + l * math.log(2.0), 0.5,
                              size=(n, 3)).astype(np.float32)
        quats = r.normal(0.0, 1.0, size=(n, 4)).astype(np.float32)
        logits = r.normal(1.0, 1.0, size=(n,)).astype(np.float32)
        sh = r.standard_normal(size=(n, SH_COEFFS, 3), dtype=np.float32)
        sh *= np.float32(sh_std)
        if spatial_order:
            perm = _morton_order(means[:, 0].astype(np.float64) - x0,
                                 means[:, 1].astype(np.float64) - y0,
                                 max(x1 - x0, y1 - y0))
            means = means[perm]
            log_scales = log_scales[perm]
            quats = quats[perm]
            logits = logits[perm]
            sh = sh[perm]
        fv = 0.0 if filter_vars is None else float(filter_vars[l])
        levels.append(Level(np.ascontiguousarray(means), np.ascontiguousarray(log_scales),
                            np.ascontiguousarray(quats), np.ascontiguousarray(logits),
                            np.ascontiguousarray(sh), fv))
    cell = extent / grid
    cc = (np.arange(grid) + 0.5) * cell
    gx, gy = np.meshgrid(cc, cc, indexing="xy")   # index = j * grid + i
    centers = np.stack([gx.ravel(), gy.ravel(),
                        height(hp, gx.ravel(), gy.ravel()) + cam_height], axis=1)
    return Scene(levels=levels,
                 d_thresholds=np.asarray(d_thresholds[:num_levels - 1], np.float64),
                 chunk_centers=centers.astype(np.float64), sh_degree=3,
                 extent=float(extent), height_params=hp)


def catmull_rom_trajectory(seed: int, n_poses: int, lo: float, hi: float,
                           n_ctrl: int = 8) -> np.ndarray:
    """(n_poses, 2) positions spaced uniformly in arc length along a
    Catmull-Rom spline through ``n_ctrl`` seeded control points in
    [lo, hi]^2."""
    r = _rng(seed, 200)
    P = r.uniform(lo, hi, size=(n_ctrl, 2))
    Pe = np.concatenate([2 * P[:1] - P[1:2], P, 2 * P[-1:] - P[-2:-1]], axis=0)
    dense = []
    m = 256
    for i in range(1, n_ctrl):
        p0, p1, p2, p3 = Pe[i - 1], Pe[i], Pe[i + 1], Pe[i + 2]
        s = np.linspace(0.0, 1.0, m, endpoint=(i == n_ctrl - 1))[:, None]
        seg = 0.5 * ((2 * p1) + (-p0 + p2) * s + (2 * p0 - 5 * p1 + 4 * p2 - p3) * s ** 2
                     + (-p0 + 3 * p1 - 3 * p2 + p3) * s ** 3)
        dense.append(seg)
    dense = np.concatenate(dense, axis=0)
    seglen = np.linalg.norm(np.diff(dense, axis=0), axis=1)
    arc = np.concatenate([[0.0], np.cumsum(seglen)])
    targets = np.linspace(0.0, arc[-1], n_poses)
    xs = np.interp(targets, arc, dense[:, 0])
    ys = np.interp(targets, arc, dense[:, 1])
    return np.stack([xs, ys], axis=1)


def outdoor_trajectory(scene: Scene, seed: int = 0, n_poses: int = 300,
                       width: int = 1920, height_px: int = 1080,
                       fov_y_deg: float = 70.0, cam_height: float = 2.0,
                       pitch_deg: float = 10.0, margin: float = 0.1) -> List[Camera]:
    """Street-level cameras along a seeded spline, ``cam_height`` above the
    heightfield, looking along the path tangent pitched ``pitch_deg`` down."""
    E = scene.extent
    xy = catmull_rom_trajectory(seed, n_poses, margin * E, (1 - margin) * E)
    tang = np.gradient(xy, axis=0)
    cams = []
    pitch = math.radians(pitch_deg)
    for i in range(n_poses):
        tx, ty = tang[i]
        nrm = math.hypot(tx, ty) or 1.0
        fx_, fy_ = tx / nrm, ty / nrm
        pz = float(height(scene.height_params, xy[i, 0], xy[i, 1])) + cam_height
        fwd = (fx_ * math.cos(pitch), fy_ * math.cos(pitch), -math.sin(pitch))
        cams.append(look_at((xy[i, 0], xy[i, 1], pz), fwd, (0.0, 0.0, 1.0),
                            width, height_px, fov_y_deg))
    return cams


def random_street_cameras(scene: Scene, seed: int, n: int, width: int, height_px: int,
                          fov_y_deg: float = 70.0, cam_height: float = 2.0,
                          pitch_deg: float = 10.0, inner: float = 0.8) -> List[Camera]:
    """Uniform positions in the inner ``inner`` fraction of the world,
    uniform yaw, fixed downward pitch."""
    r = _rng(seed, 300)
    E = scene.extent
    lo, hi = (1 - inner) / 2 * E, (1 + inner) / 2 * E
    cams = []
    pitch = math.radians(pitch_deg)
    for _ in range(n):
        x, y = r.uniform(lo, hi, size=2)
        yaw = r.uniform(0, 2 * math.pi)
        pz = float(height(scene.height_params, x, y)) + cam_height
        fwd = (math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), -math.sin(pitch))
        cams.append(look_at((x, y, pz), fwd, (0.0, 0.0, 1.0), width, height_px, fov_y_deg))
    return cams


def chunk_views(scene: Scene, chunk: int, seed: int, n: int, width: int, height_px: int,
                fov_y_deg: float = 70.0, cam_height: float = 2.0,
                pitch_deg: float = 10.0) -> List[Camera]:
    """Views of one chunk of a square chunk grid (index j * grid + i): uniform
    positions inside the chunk's cell at street height, uniform yaw, fixed
    downward pitch -- camera positions within the chunk with random
    orientations, as the visibility filtering of Sec. 3 uses."""
    r = _rng(seed, 310 + chunk)
    K = scene.chunk_centers.shape[0]
    grid = int(round(math.sqrt(K)))
    cell = scene.extent / grid
    i, j = chunk % grid, chunk // grid
    pitch = math.radians(pitch_deg)
    cams = []
    for _ in range(n):
        x = r.uniform(i * cell, (i + 1) * cell)
        y = r.uniform(j * cell, (j + 1) * cell)
        yaw = r.uniform(0, 2 * math.pi)
        pz = float(height(scene.height_params, x, y)) + cam_height
        fwd = (math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), -math.sin(pitch))
        cams.append(look_at((x, y, pz), fwd, (0.0, 0.0, 1.0), width, height_px, fov_y_deg))
    return cams


def kmeans_init(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct seeded indices into n positions (initial K-means centres)."""
    return _rng(seed, 320).choice(n, size=k, replace=False).astype(np.int32)


def camera_positions(cams: Sequence[Camera]) -> np.ndarray:
    return np.array([np.asarray(c.center, np.float64) for c in cams])


def finetune_scene(seed: int = 0, n: int = 2_000_000, cell: float = 62.5,
                   center_xy=(500.0, 500.0)) -> Scene:
    """One chunk cell of the outdoor generator (level-0 density scaled so
    the cell holds ``n`` Gaussians)."""
    cx, cy = center_xy
    region = (cx - cell / 2, cy - cell / 2, cx + cell / 2, cy + cell / 2)
    return outdoor_scene(seed=seed, n0=n, num_levels=1, extent=1000.0, grid=16,
                         d_thresholds=(), region=region)


def perturb_scene(scene: Scene, seed: int, mean_std: float = 0.05,
                  logit_std: float = 0.3) -> Scene:
    """Copy of ``scene`` with means + N(0, mean_std) and opacity logits +
    N(0, logit_std) (the fine-tuning target)."""
    r = _rng(seed, 400)
    levels = []
    for l in scene.levels:
        levels.append(dataclasses.replace(
            l,
            means=(l.means + r.normal(0, mean_std, size=l.means.shape)).astype(np.float32),
            opacity_logits=(l.opacity_logits + r.normal(0, logit_std, size=l.opacity_logits.shape)).astype(np.float32)))
    return dataclasses.replace(scene, levels=levels)


def finetune_cameras(scene: Scene, seed: int = 0, n: int = 32, width: int = 1280,
                     height_px: int = 720, cell: float = 62.5, center_xy=(500.0, 500.0),
                     fov_y_deg: float = 70.0) -> List[Camera]:
    """Street-height views placed around the cell, looking inward."""
    r = _rng(seed, 500)
    cx, cy = center_xy
    cams = []
    for _ in range(n):
        ang = r.uniform(0, 2 * math.pi)
        rad = r.uniform(0.3, 0.6) * cell
        x, y = cx + rad * math.cos(ang), cy + rad * math.sin(ang)
        yaw = ang + math.pi + r.uniform(-0.4, 0.4)
        pz = float(height(scene.height_params, x, y)) + 2.0
        pitch = math.radians(r.uniform(5.0, 20.0))
        fwd = (math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), -math.sin(pitch))
        cams.append(look_at((x, y, pz), fwd, (0.0, 0.0, 1.0), width, height_px, fov_y_deg))
    return cams


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def workload_plain(seed: int = 0):
    """4,096-Gaussian single-level scene, one 256x256 camera, 60 deg FOV."""
    return plain_scene(seed), [plain_camera()]


def workload_outdoor(seed: int = 0, n_poses: int = 300, scale: float = 1.0,
                     width: int = 1920, height_px: int = 1080):
    """Outdoor LOD scene, 16M/4M/1M/250k Gaussians over 1 km^2, 16x16 chunk
    grid, 300-pose street-level trajectory at 1920x1080, 70 deg vertical FOV.
    ``scale`` < 1 shrinks the world side by sqrt(scale) at constant density
    (and the chunk grid with it) for oracle-sized tests."""
    side = 1000.0 * math.sqrt(scale)
    grid = max(1, int(round(16 * math.sqrt(scale))))
    scene = outdoor_scene(seed=seed, n0=int(16_000_000 * scale), num_levels=4,
                          extent=side, grid=grid)
    cams = outdoor_trajectory(scene, seed=seed, n_poses=n_poses, width=width,
                              height_px=height_px)
    return scene, cams


# --------------------------------------------------------------------------
# large indoor + outdoor scene
# --------------------------------------------------------------------------
def _room_surface_points(r: np.random.Generator, n: int, x0: float, y0: float, side: float,
                         room: float, spacing: float, hp: dict):
    """n points uniform on the faces of room-sized boxes laid out on a grid of
    pitch `spacing` inside the square [x0, x0 + side]^2 (floors on the
    heightfield): floor, ceiling and four walls, all of equal area."""
    per = int(side // spacing)
    k = r.integers(0, per * per, size=n)
    cx = x0 + (k % per + 0.5) * spacing
    cy = y0 + (k // per + 0.5) * spacing
    face = r.integers(0, 6, size=n)
    u = r.uniform(-0.5, 0.5, size=n) * room
    v = r.uniform(-0.5, 0.5, size=n) * room
    half = 0.5 * room
    base = height(hp, cx, cy)
    x = np.where(face == 2, cx - half, np.where(face == 3, cx + half, cx + u))
    y = np.where(face == 4, cy - half, np.where(face == 5, cy + half,
                                                np.where(face < 2, cy + v, cy + u)))
    z = np.where(face == 0, base, np.where(face == 1, base + room, base + half + v))
    return x, y, z


def large_scene(seed: int = 0, n0: int = 60_000_000, num_levels: int = 6, extent: float = 1000.0,
                grid: int = 32, indoor_fraction: float = 0.25,
                d_thresholds: Sequence[float] = (10.0, 20.0, 40.0, 80.0, 160.0),
                log_scale_mean0: float = math.log(0.125), jitter0: float = 0.5,
                sh_std: float = 0.2, cam_height: float = 2.0) -> Scene:
    """Outdoor heightfield world with an indoor quadrant: level l holds
    n0 / 4^l Gaussians, of which `indoor_fraction` sit on the faces of 10 m
    rooms (20 m pitch) filling the quadrant [0, extent/2]^2 and the rest on
    the terrain as in outdoor_scene.  Chunk grid grid x grid."""
    hp = height_params(seed)
    levels = []
    for l in range(num_levels):
        n = max(int(n0 // (4 ** l)), 1)
        n_in = int(n * indoor_fraction)
        n_out = n - n_in
        r = _rng(seed, 11, l)
        ox = r.uniform(0.0, extent, size=n_out)
        oy = r.uniform(0.0, extent, size=n_out)
        oz = height(hp, ox, oy)
        ix, iy, iz = _room_surface_points(r, n_in, 0.0, 0.0, extent / 2, 10.0, 20.0, hp)
        x = np.concatenate([ox, ix]); y = np.concatenate([oy, iy]); z = np.concatenate([oz, iz])
        del ox, oy, oz, ix, iy, iz
        jit = r.normal(0.0, jitter0 * 2.0 ** l, size=(n, 3))
        means = np.empty((n, 3), np.float32)
        means[:, 0] = x + jit[:, 0]
        means[:, 1] = y + jit[:, 1]
        means[:, 2] = z + jit[:, 2]
        del x, y, z, jit
        log_scales = r.normal(log_scale_mean0 + l * math.log(2.0), 0.5, size=(n, 3)).astype(np.float32)
        quats = r.normal(0.0, 1.0, size=(n, 4)).astype(np.float32)
        logits = r.normal(1.0, 1.0, size=(n,)).astype(np.float32)
        sh = r.standard_normal(size=(n, SH_COEFFS, 3), dtype=np.float32)
        sh *= np.float32(sh_std)
        perm = _morton_order(means[:, 0].astype(np.float64), means[:, 1].astype(np.float64), extent)
        levels.append(Level(np.ascontiguousarray(means[perm]), np.ascontiguousarray(log_scales[perm]),
                            np.ascontiguousarray(quats[perm]), np.ascontiguousarray(logits[perm]),
                            np.ascontiguousarray(sh[perm]), 0.0))
        del means, log_scales, quats, logits, sh, perm
    cell = extent / grid
    cc = (np.arange(grid) + 0.5) * cell
    gx, gy = np.meshgrid(cc, cc, indexing="xy")
    centers = np.stack([gx.ravel(), gy.ravel(),
                        height(hp, gx.ravel(), gy.ravel()) + cam_height], axis=1)
    return Scene(levels=levels, d_thresholds=np.asarray(d_thresholds[:num_levels - 1], np.float64),
                 chunk_centers=centers.astype(np.float64), sh_degree=3, extent=float(extent),
                 height_params=hp)


def workload_large(seed: int = 0, n_cams: int = 64, scale: float = 1.0, width: int = 3840,
                   height_px: int = 2160):
    """60M level-0 Gaussians over 6 levels (indoor quadrant + outdoor), 32x32
    chunks, a batch of n_cams street-height cameras at 3840x2160.  ``scale``
    shrinks the world at constant density."""
    side = 1000.0 * math.sqrt(scale)
    grid = max(1, int(round(32 * math.sqrt(scale))))
    scene = large_scene(seed=seed, n0=int(60_000_000 * scale), extent=side, grid=grid)
    cams = random_street_cameras(scene, seed + 5, n_cams, width, height_px)
    return scene, cams
