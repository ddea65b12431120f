"""Seeded synthetic point clouds (inputs only; no clustering arithmetic here).

The paper's own data (KITTI odometry / semanticKITTI scans after ground removal,
Section 3.4) is not available, so these generators stand in for it.  Every
coordinate is a float32 multiple of 1/1024 m, and every cloud is shuffled
with its seed: the paper makes its synthetic clouds unorganised by randomising
the point index (Section 3.3.1).

Workloads
---------
``blobs_20k``      20,000 points in a 40 m cube: 50 isotropic Gaussian blobs
                   (sigma 0.3-1.5 m, 360 points each) plus 2,000 uniform noise
                   points; d = 0.5, min 1, max inf; seed 1.
``frame_120k``     one 64-beam rotating-LiDAR frame: flat ground to 80 m, 200
                   boxes/cylinders (0.5-5 m) at random poses, 2 cm range noise;
                   ~120k points; d = 0.35, min 50, max 50,000; seed 2.
``map_27m``        230 such frames along a straight 2 km corridor (sensor every
                   8.7 m) with buildings, poles and vehicles; ~27M points;
                   d = 0.2, min 100, max 2,000,000; seed 3.
``batch_256``      256 frames, n log-uniform in [20k, 180k], d per frame from
                   {0.25, 0.35, 0.5}, min 50, max 50,000; seed 4.
``serve``          request clouds of 10k-2M points (log-uniform); single
                   frames up to 180k, larger ones cut from consecutive corridor
                   frames; d ~ U[0.15, 0.6], min ~ U{10..200}, max inf; seed 5.
``voxel_clusters`` the paper's synthetic recipe (Section 3.3.1): m points filled
                   evenly into n random voxels, optionally shifted by a Gaussian
                   of std sigma, index shuffled.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

INF_SIZE = (1 << 63) - 1

SENSOR_HEIGHT = 1.73
N_BEAMS = 64
ELEV_TOP_DEG = 2.0
ELEV_BOTTOM_DEG = -24.8
MAX_RANGE = 80.0
RANGE_NOISE = 0.02


@dataclass
class Cloud:
    xyz: np.ndarray  # float32 [n, 3], multiples of 1/1024
    d: float
    min_size: int
    max_size: int
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


def to_grid(x: np.ndarray) -> np.ndarray:
    """Round generated coordinates to float32 multiples of 1/1024 m."""
    return (np.rint(np.asarray(x, dtype=np.float64) * 1024.0) / 1024.0).astype(np.float32)


def _shuffle(rng: np.random.Generator, xyz: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(xyz[rng.permutation(xyz.shape[0])])


# --------------------------------------------------------------------------
# Blobs
# --------------------------------------------------------------------------

def blobs(seed: int = 1, n_blobs: int = 50, per_blob: int = 360, n_noise: int = 2000,
          cube: float = 40.0, sigma=(0.3, 1.5)) -> np.ndarray:
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, cube, size=(n_blobs, 3))
    sig = rng.uniform(sigma[0], sigma[1], size=n_blobs)
    pts = [centres[b] + rng.normal(0.0, sig[b], size=(per_blob, 3)) for b in range(n_blobs)]
    pts.append(rng.uniform(0.0, cube, size=(n_noise, 3)))
    xyz = to_grid(np.concatenate(pts, axis=0))
    return _shuffle(rng, xyz)


def blobs_20k(seed: int = 1) -> Cloud:
    return Cloud(blobs(seed), 0.5, 1, INF_SIZE, "blobs_20k")


# --------------------------------------------------------------------------
# Ray casting against a ground plane, oriented boxes and vertical cylinders
# --------------------------------------------------------------------------

@dataclass
class Scene:
    # boxes: rows (cx, cy, z0, length, width, height, yaw); base at z = z0
    boxes: np.ndarray
    # cylinders: rows (cx, cy, z0, radius, height); base at z = z0
    cyls: np.ndarray


def random_scene(rng: np.random.Generator, n_objects: int = 200, radius: float = 75.0,
                 size=(0.5, 5.0)) -> Scene:
    """Objects at random poses in a disc around the origin (sensor-centred)."""
    kind = rng.random(n_objects) < 0.6
    nb, nc = int(kind.sum()), int((~kind).sum())
    r = np.sqrt(rng.uniform((4.0 / radius) ** 2, 1.0, size=n_objects)) * radius
    th = rng.uniform(0, 2 * math.pi, size=n_objects)
    cx, cy = r * np.cos(th), r * np.sin(th)
    # about half of the objects rest on the ground, the rest float up to 0.6 m
    z0 = np.where(rng.random(n_objects) < 0.5, 0.0, rng.uniform(0.1, 0.6, n_objects))
    boxes = np.stack([cx[kind], cy[kind], z0[kind], rng.uniform(*size, nb),
                      rng.uniform(*size, nb), rng.uniform(*size, nb),
                      rng.uniform(0, math.pi, nb)], axis=1)
    cyls = np.stack([cx[~kind], cy[~kind], z0[~kind],
                     rng.uniform(size[0] / 2, size[1] / 2, nc), rng.uniform(*size, nc)], axis=1)
    return Scene(boxes, cyls)


def corridor_scene(rng: np.random.Generator, length: float = 2000.0) -> Scene:
    """Buildings (boxes) along both sides, poles (cylinders), vehicles (boxes)."""
    boxes, cyls = [], []
    for side in (-1.0, 1.0):
        x = -60.0
        while x < length + 60.0:
            L = rng.uniform(10.0, 40.0)
            depth = rng.uniform(8.0, 20.0)
            setback = rng.uniform(9.0, 15.0)
            boxes.append((x + L / 2, side * (setback + depth / 2), 0.0, L, depth,
                          rng.uniform(5.0, 25.0), 0.0))
            x += L + rng.uniform(2.0, 15.0)
        x = -60.0 + rng.uniform(0, 20.0)
        while x < length + 60.0:
            cyls.append((x, side * rng.uniform(6.0, 7.0), 0.0, rng.uniform(0.1, 0.25),
                         rng.uniform(4.0, 9.0)))
            x += rng.uniform(15.0, 40.0)
    n_veh = int(length / 5.0)
    for _ in range(n_veh):
        # vehicles have 0.25-0.4 m of ground clearance
        boxes.append((rng.uniform(-50.0, length + 50.0), rng.uniform(-4.5, 4.5),
                      rng.uniform(0.25, 0.4), rng.uniform(3.5, 5.5), rng.uniform(1.6, 2.0),
                      rng.uniform(1.0, 1.6), rng.normal(0.0, 0.05)))
    return Scene(np.asarray(boxes, dtype=np.float64), np.asarray(cyls, dtype=np.float64))


def _ray_box(ox, oy, oz, dx, dy, dz, b):
    cx, cy, z0, L, W, H, yaw = b
    c, s = math.cos(yaw), math.sin(yaw)
    lx, ly = ox - cx, oy - cy
    px, py = c * lx + s * ly, -s * lx + c * ly
    ux, uy = c * dx + s * dy, -s * dx + c * dy
    tmin = np.full(ux.shape, -np.inf)
    tmax = np.full(ux.shape, np.inf)
    for p, u, lo, hi in ((px, ux, -L / 2, L / 2), (py, uy, -W / 2, W / 2), (oz, dz, z0, z0 + H)):
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / u
            t1 = (lo - p) * inv
            t2 = (hi - p) * inv
        par = u == 0
        inside = (p >= lo) & (p <= hi)
        t1 = np.where(par, np.where(inside, -np.inf, np.inf), t1)
        t2 = np.where(par, np.where(inside, np.inf, -np.inf), t2)
        tmin = np.maximum(tmin, np.minimum(t1, t2))
        tmax = np.minimum(tmax, np.maximum(t1, t2))
    hit = (tmin <= tmax) & (tmin > 0)
    return np.where(hit, tmin, np.inf)


def _ray_cyl(ox, oy, oz, dx, dy, dz, cyl):
    cx, cy, z0, R, H = cyl
    lx, ly = ox - cx, oy - cy
    a = dx * dx + dy * dy
    b = 2 * (lx * dx + ly * dy)
    cc = lx * lx + ly * ly - R * R
    disc = b * b - 4 * a * cc
    out = np.full(dx.shape, np.inf)
    ok = (disc >= 0) & (a > 0)
    with np.errstate(invalid="ignore", divide="ignore"):
        t1 = (-b - np.sqrt(np.where(ok, disc, 0))) / (2 * np.where(ok, a, 1))
    z1 = oz + t1 * dz
    side = ok & (t1 > 0) & (z1 >= z0) & (z1 <= z0 + H)
    out = np.where(side, t1, out)
    with np.errstate(invalid="ignore", divide="ignore"):
        tt = (z0 + H - oz) / dz
    xt, yt = lx + tt * dx, ly + tt * dy
    top = (dz != 0) & (tt > 0) & (xt * xt + yt * yt <= R * R)
    return np.where(top, np.minimum(out, tt), out)


def lidar_frame(rng: np.random.Generator, scene: Scene, sensor=(0.0, 0.0), n_az: int = 1925,
                max_range: float = MAX_RANGE) -> np.ndarray:
    """One 64-beam scan from (sensor, SENSOR_HEIGHT); float64 [m, 3] hits."""
    sx, sy = sensor
    sz = SENSOR_HEIGHT
    elev = np.deg2rad(np.linspace(ELEV_TOP_DEG, ELEV_BOTTOM_DEG, N_BEAMS))
    az = (np.arange(n_az) + rng.uniform(0, 1)) * (2 * math.pi / n_az)
    ce, se = np.cos(elev)[:, None], np.sin(elev)[:, None]
    DX = ce * np.cos(az)[None, :]
    DY = ce * np.sin(az)[None, :]
    DZ = np.broadcast_to(se, DX.shape).copy()
    # ground plane z = 0, hits within max_range horizontally
    with np.errstate(divide="ignore"):
        tg = np.where(DZ < 0, -sz / DZ, np.inf)
    tg = np.where(tg * ce <= max_range, tg, np.inf)
    T = tg.copy()

    def window(cx, cy, rb):
        rx, ry = cx - sx, cy - sy
        rho = math.hypot(rx, ry)
        if rho - rb > max_range:
            return None
        if rho <= rb:
            return np.arange(n_az)
        half = math.asin(min(1.0, rb / rho)) + 2 * math.pi / n_az
        th = math.atan2(ry, rx)
        lo = int(math.floor((th - half) / (2 * math.pi) * n_az))
        hi = int(math.ceil((th + half) / (2 * math.pi) * n_az))
        return np.arange(lo, hi + 1) % n_az

    for b in scene.boxes:
        cols = window(b[0], b[1], 0.5 * math.hypot(b[3], b[4]))
        if cols is None:
            continue
        t = _ray_box(sx, sy, sz, DX[:, cols], DY[:, cols], DZ[:, cols], b)
        T[:, cols] = np.minimum(T[:, cols], t)
    for c in scene.cyls:
        cols = window(c[0], c[1], c[3])
        if cols is None:
            continue
        t = _ray_cyl(sx, sy, sz, DX[:, cols], DY[:, cols], DZ[:, cols], c)
        T[:, cols] = np.minimum(T[:, cols], t)

    T = np.where(T * ce <= max_range, T, np.inf)
    hit = np.isfinite(T)
    t = T[hit] + rng.normal(0.0, RANGE_NOISE, size=int(hit.sum()))
    pts = np.stack([sx + t * DX[hit], sy + t * DY[hit], sz + t * DZ[hit]], axis=1)
    return pts


def frame_120k(seed: int = 2) -> Cloud:
    rng = np.random.default_rng(seed)
    scene = random_scene(rng, 200)
    xyz = to_grid(lidar_frame(rng, scene, n_az=1925))
    return Cloud(_shuffle(rng, xyz), 0.35, 50, 50_000, "frame_120k")


def frame_of_size(rng: np.random.Generator, n: int) -> np.ndarray:
    """A frame-generator scan cut to exactly n points (random subset)."""
    n_az = max(64, int(math.ceil(n * 1.25 / 55.0)))
    while True:
        scene = random_scene(rng, 200)
        pts = lidar_frame(rng, scene, n_az=n_az)
        if pts.shape[0] >= n:
            sel = rng.choice(pts.shape[0], size=n, replace=False)
            return pts[np.sort(sel)]
        n_az = int(n_az * 1.3) + 1


# --------------------------------------------------------------------------
# Accumulated corridor map
# --------------------------------------------------------------------------

MAP_FRAMES = 230
MAP_SPACING = 8.7


def corridor_frames(seed: int, n_frames: int = MAP_FRAMES, spacing: float = MAP_SPACING,
                    n_az: int = 1925, first: int = 0):
    """Yield float64 hit arrays of consecutive frames along the corridor."""
    rng = np.random.default_rng(seed)
    scene = corridor_scene(rng, length=max(2000.0, (first + n_frames) * spacing))
    for k in range(first, first + n_frames):
        frng = np.random.default_rng([seed, k])
        yield lidar_frame(frng, scene, sensor=(k * spacing, 0.0), n_az=n_az)


def map_27m(seed: int = 3, n_frames: int = MAP_FRAMES) -> Cloud:
    parts = [to_grid(p) for p in corridor_frames(seed, n_frames)]
    xyz = np.concatenate(parts, axis=0)
    rng = np.random.default_rng([seed, 1 << 20])
    return Cloud(_shuffle(rng, xyz), 0.2, 100, 2_000_000, "map_27m",
                 {"frames": n_frames})


def map_crop(cloud: Cloud, x_lo: float, x_hi: float) -> Cloud:
    """Points of an accumulated map with x in [x_lo, x_hi), original order kept."""
    m = (cloud.xyz[:, 0] >= x_lo) & (cloud.xyz[:, 0] < x_hi)
    return Cloud(np.ascontiguousarray(cloud.xyz[m]), cloud.d, cloud.min_size,
                 cloud.max_size, f"{cloud.name}[x in {x_lo:g}..{x_hi:g}]")


# --------------------------------------------------------------------------
# Batch and serving streams
# --------------------------------------------------------------------------

def batch_256(seed: int = 4, n_frames: int = 256, lo: int = 20_000, hi: int = 180_000):
    """List of Cloud, one per frame (frame-local parameters)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_frames)).astype(np.int64)
    ds = rng.choice(np.array([0.25, 0.35, 0.5]), size=n_frames)
    out = []
    for f in range(n_frames):
        frng = np.random.default_rng([seed, f])
        xyz = to_grid(frame_of_size(frng, int(sizes[f])))
        out.append(Cloud(_shuffle(frng, xyz), float(ds[f]), 50, 50_000, f"batch[{f}]"))
    return out


def serve_request(seed: int, i: int, lo: int = 10_000, hi: int = 2_000_000,
                  corridor_seed: int = 3) -> Cloud:
    """Request i of the serving stream."""
    rng = np.random.default_rng([seed, i])
    n = int(math.exp(rng.uniform(math.log(lo), math.log(hi))))
    d = float(np.float32(rng.uniform(0.15, 0.6)))
    mn = int(rng.integers(10, 201))
    if n <= 180_000:
        pts = frame_of_size(rng, n)
    else:
        per = 115_000
        k = int(math.ceil(n / per)) + 1
        first = int(rng.integers(0, MAP_FRAMES))
        pts = np.concatenate(list(corridor_frames(corridor_seed, k, first=first)), axis=0)
        sel = rng.choice(pts.shape[0], size=min(n, pts.shape[0]), replace=False)
        pts = pts[np.sort(sel)]
    xyz = to_grid(pts)
    return Cloud(_shuffle(rng, xyz), d, mn, INF_SIZE, f"serve[{i}]")


def poisson_arrivals(seed: int, rate: float, duration: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng([seed, 7])
    gaps = rng.exponential(1.0 / rate, size=int(rate * duration * 1.5) + 16)
    t = np.cumsum(gaps)
    return t[t < duration]


# --------------------------------------------------------------------------
# The paper's synthetic recipe (Section 3.3.1)
# --------------------------------------------------------------------------

def voxel_clusters(seed: int, n_clusters: int, density: int, sigma: float = 0.0,
                   voxel: float = 1.0, grid: int = 64) -> np.ndarray:
    """m = density points filled evenly into each of n random voxels of a
    grid^3 lattice (every other lattice site, so voxels never touch), then
    shifted by N(0, sigma) per coordinate; index shuffled."""
    rng = np.random.default_rng(seed)
    sites = rng.choice((grid // 2) ** 3, size=n_clusters, replace=False)
    ix = 2 * (sites % (grid // 2))
    iy = 2 * ((sites // (grid // 2)) % (grid // 2))
    iz = 2 * (sites // (grid // 2) ** 2)
    side = max(1, int(round(density ** (1.0 / 3.0))))
    while side ** 3 < density:
        side += 1
    lin = (np.arange(side) + 0.5) / side
    cube = np.stack(np.meshgrid(lin, lin, lin, indexing="ij"), axis=-1).reshape(-1, 3)[:density]
    pts = (np.stack([ix, iy, iz], axis=1)[:, None, :] + cube[None, :, :]) * voxel
    pts = pts.reshape(-1, 3)
    if sigma > 0:
        pts = pts + rng.normal(0.0, sigma, size=pts.shape)
    return _shuffle(rng, to_grid(pts))


WORKLOADS = {"blobs_20k": blobs_20k, "frame_120k": frame_120k, "map_27m": map_27m}
