"""Seeded synthetic point clouds shaped like the paper's workloads.

This module holds no part of the decimation arithmetic: it only produces inputs.
Both the CUDA path and the CPU oracle read the same arrays it returns.

The paper's own inputs (a RealSense D435 corridor and a simulated Gazebo office,
arXiv 2102.11084 Sec. II-D/E) are not available, so these generators stand in for
them:

* ``rgbd_frame``  -- a depth camera frame back-projected through a pinhole model
  (fx = fy = 525, principal point at the image centre), of a scene of 6 random
  planes and 20 random axis-aligned boxes between 0.5 m and 5 m, with depth noise
  sigma = 0.002 z^2 and exactly round(nan_frac * W * H) pixels forced to NaN (plus
  the pixels whose ray hits nothing).  Row-major pixel order.
* ``fused_map``   -- a large unordered map cloud: 70 % of the points on 8 random
  planes and 400 random boxes inside a 40 x 40 x 10 m volume (allocated by area,
  isotropic noise sigma = 5 mm), 30 % uniform clutter, exactly round(2 %) NaN rows,
  then a global seeded shuffle.
* ``batch_frames`` -- 64 frames of uneven size (each a seeded subset, in pixel
  order, of a 1280 x 720 frame) with a per-frame leaf from {0.02, 0.05, 0.1} m.
* ``serving_trace`` -- Poisson arrivals of 640 x 480 frames from many sensors.
* ``sensor_poses`` -- camera-to-map poses [R|t] of a depth camera on a mobile robot
  (optical axis horizontal, random heading, lens 0.8-1.2 m above the floor, position
  inside the 40 x 40 m map) and the height band kept in the map frame.

All randomness comes from numpy's PCG64 with explicit seeds.
"""
from __future__ import annotations

from typing import NamedTuple

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _random_unit(rng: np.random.Generator, k: int) -> np.ndarray:
    v = rng.normal(size=(k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def rgbd_frame(width: int = 640, height: int = 480, seed: int = 0, *, fx: float = 525.0,
               fy: float = 525.0, cx: float | None = None, cy: float | None = None,
               n_planes: int = 6, n_boxes: int = 20, z_min: float = 0.5, z_max: float = 5.0,
               nan_frac: float = 0.1) -> np.ndarray:
    """One back-projected RGB-D frame as float32 [height*width, 3] (NaN = no depth)."""
    rng = _rng(seed)
    cx = (width - 1) / 2.0 if cx is None else cx
    cy = (height - 1) / 2.0 if cy is None else cy
    u = np.arange(width, dtype=np.float64)
    v = np.arange(height, dtype=np.float64)
    dx = np.broadcast_to(((u - cx) / fx)[None, :], (height, width)).reshape(-1)
    dy = np.broadcast_to(((v - cy) / fy)[:, None], (height, width)).reshape(-1)
    best = np.full(dx.shape, np.inf)

    def random_ray_point(depth):
        pu = rng.uniform(0, width)
        pv = rng.uniform(0, height)
        return np.array([(pu - cx) / fx * depth, (pv - cy) / fy * depth, depth])

    # planes: n . x = off;  plane 0 is fronto-parallel at the back of the scene
    for k in range(n_planes):
        if k == 0:
            n = np.array([0.0, 0.0, 1.0])
            off = rng.uniform(z_max - 0.5, z_max)
        else:
            n = _random_unit(rng, 1)[0]
            off = float(n @ random_ray_point(rng.uniform(1.0, z_max)))
        denom = n[0] * dx + n[1] * dy + n[2]
        with np.errstate(divide="ignore", invalid="ignore"):
            t = off / denom
        hit = (t >= z_min) & (t <= z_max)
        np.minimum(best, np.where(hit, t, np.inf), out=best)

    # axis-aligned boxes: slab test; depth along the ray is t (d_z = 1)
    for _ in range(n_boxes):
        c = random_ray_point(rng.uniform(1.0, z_max - 0.5))
        h = rng.uniform(0.05, 0.4, size=3)
        lo, hi = c - h, c + h
        with np.errstate(divide="ignore", invalid="ignore"):
            t0x, t1x = lo[0] / dx, hi[0] / dx
            t0y, t1y = lo[1] / dy, hi[1] / dy
        tnear = np.maximum(np.minimum(t0x, t1x), np.minimum(t0y, t1y))
        tfar = np.minimum(np.maximum(t0x, t1x), np.maximum(t0y, t1y))
        tnear = np.maximum(tnear, lo[2])
        tfar = np.minimum(tfar, hi[2])
        hit = (tnear <= tfar) & (tnear >= z_min) & (tnear <= z_max)
        np.minimum(best, np.where(hit, tnear, np.inf), out=best)

    z = best
    has = np.isfinite(z)
    z = np.where(has, z + rng.normal(size=z.shape) * (0.002 * np.where(has, z, 0.0) ** 2), np.nan)
    pts = np.stack([z * dx, z * dy, z], axis=1).astype(np.float32)
    n_nan = int(round(nan_frac * width * height))
    if n_nan:
        pts[rng.permutation(width * height)[:n_nan]] = np.nan
    return pts


def _plane_points(rng, n_pts, normal, point, ext, batch=1 << 20):
    """Uniform samples on the plane (normal, point) clipped to the box [0, ext]."""
    a = int(np.argmax(np.abs(normal)))
    b, c = [i for i in range(3) if i != a]
    out = []
    got = 0
    while got < n_pts:
        m = max(1024, min(batch, 2 * (n_pts - got)))
        s = np.empty((m, 3))
        s[:, b] = rng.uniform(0, ext[b], m)
        s[:, c] = rng.uniform(0, ext[c], m)
        s[:, a] = point[a] - (normal[b] * (s[:, b] - point[b]) +
                              normal[c] * (s[:, c] - point[c])) / normal[a]
        s = s[(s[:, a] >= 0) & (s[:, a] <= ext[a])]
        out.append(s[: n_pts - got])
        got += out[-1].shape[0]
    return np.concatenate(out) if out else np.zeros((0, 3))


def _plane_area(rng, normal, point, ext, trials=20000):
    a = int(np.argmax(np.abs(normal)))
    b, c = [i for i in range(3) if i != a]
    sb = rng.uniform(0, ext[b], trials)
    sc = rng.uniform(0, ext[c], trials)
    sa = point[a] - (normal[b] * (sb - point[b]) + normal[c] * (sc - point[c])) / normal[a]
    frac = np.mean((sa >= 0) & (sa <= ext[a]))
    return frac * ext[b] * ext[c] / abs(normal[a])


def _box_points(rng, n_pts, lo, hi):
    e = hi - lo
    faces = np.array([e[1] * e[2], e[1] * e[2], e[0] * e[2], e[0] * e[2], e[0] * e[1], e[0] * e[1]])
    which = rng.choice(6, size=n_pts, p=faces / faces.sum())
    s = lo + rng.uniform(size=(n_pts, 3)) * e
    axis = which // 2
    side = which % 2
    s[np.arange(n_pts), axis] = np.where(side == 1, hi[axis], lo[axis])
    return s


def fused_map(n: int = 50_000_000, seed: int = 0, *, extent=(40.0, 40.0, 10.0), n_planes: int = 8,
              n_boxes: int = 400, surface_frac: float = 0.7, sigma: float = 0.005,
              nan_frac: float = 0.02, shuffle: bool = True) -> np.ndarray:
    """A fused, unordered map cloud as float32 [n, 3]."""
    rng = _rng(seed)
    ext = np.asarray(extent, np.float64)
    planes = []
    for _ in range(n_planes):
        nrm = _random_unit(rng, 1)[0]
        pt = rng.uniform(size=3) * ext
        planes.append((nrm, pt, _plane_area(rng, nrm, pt, ext)))
    boxes = []
    for _ in range(n_boxes):
        e = rng.uniform(0.2, 3.0, size=3)
        e = np.minimum(e, ext)
        lo = rng.uniform(size=3) * (ext - e)
        hi = lo + e
        boxes.append((lo, hi, 2 * (e[0] * e[1] + e[1] * e[2] + e[0] * e[2])))
    areas = np.array([p[2] for p in planes] + [b[2] for b in boxes])
    n_surf = int(round(surface_frac * n))
    alloc = rng.multinomial(n_surf, areas / areas.sum())
    out = np.empty((n, 3), np.float32)
    pos = 0
    for k, (nrm, pt, _) in enumerate(planes):
        m = int(alloc[k])
        if m:
            out[pos:pos + m] = _plane_points(rng, m, nrm, pt, ext)
            pos += m
    for k, (lo, hi, _) in enumerate(boxes):
        m = int(alloc[n_planes + k])
        if m:
            out[pos:pos + m] = _box_points(rng, m, lo, hi)
            pos += m
    # isotropic surface noise, in chunks to bound the temporaries
    for s in range(0, pos, 1 << 22):
        e = min(pos, s + (1 << 22))
        out[s:e] += (rng.normal(size=(e - s, 3)) * sigma).astype(np.float32)
    for s in range(pos, n, 1 << 22):
        e = min(n, s + (1 << 22))
        out[s:e] = (rng.uniform(size=(e - s, 3)) * ext).astype(np.float32)
    n_nan = int(round(nan_frac * n))
    if n_nan:
        out[rng.permutation(n)[:n_nan]] = np.nan
    if shuffle:
        out = out[rng.permutation(n)]
    return out


class BatchSpec(NamedTuple):
    frames: list            # list of float32 [N_f, 3]
    leaves: np.ndarray      # float32 [F]


def batch_frames(n_frames: int = 64, seed: int = 1, *, width: int = 1280, height: int = 720,
                 n_min: int = 20_000, n_max: int | None = None,
                 leaf_choices=(0.02, 0.05, 0.1), frame_seed_base: int = 1000) -> BatchSpec:
    """Frames of uneven size: frame f keeps a seeded subset (pixel order) of a frame."""
    rng = _rng(seed)
    n_max = width * height if n_max is None else n_max
    sizes = rng.integers(n_min, n_max, endpoint=True, size=n_frames)
    leaves = rng.choice(np.asarray(leaf_choices, np.float32), size=n_frames)
    frames = []
    for f in range(n_frames):
        full = rgbd_frame(width, height, seed=frame_seed_base + f)
        keep = np.sort(_rng(frame_seed_base + f + 7_777_777).choice(
            full.shape[0], int(sizes[f]), replace=False))
        frames.append(np.ascontiguousarray(full[keep]))
    return BatchSpec(frames, leaves.astype(np.float32))


class Request(NamedTuple):
    stream: int
    arrival_s: float
    frame: int


def serving_trace(n_streams: int = 16, rate_hz: float = 30.0, duration_s: float = 10.0,
                  pool: int = 64, seed: int = 5) -> list:
    """Poisson arrivals (seeded exponential gaps) of frames drawn from a frame pool."""
    rng = _rng(seed)
    reqs = []
    for s in range(n_streams):
        t = 0.0
        while True:
            t += float(rng.exponential(1.0 / rate_hz))
            if t >= duration_s:
                break
            reqs.append(Request(s, t, int(rng.integers(pool))))
    reqs.sort(key=lambda r: (r.arrival_s, r.stream))
    return reqs


def random_cloud(n: int, seed: int = 0, *, extent: float = 2.0, nan_frac: float = 0.05,
                 inf_frac: float = 0.0, clusters: int = 0, cluster_sigma: float = 0.01,
                 offset=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Small test clouds: uniform (or clustered) points with NaN/Inf rows."""
    rng = _rng(seed)
    if clusters:
        centres = rng.uniform(0, extent, size=(clusters, 3))
        pick = rng.integers(clusters, size=n)
        pts = centres[pick] + rng.normal(size=(n, 3)) * cluster_sigma
    else:
        pts = rng.uniform(0, extent, size=(n, 3))
    pts = (pts + np.asarray(offset)).astype(np.float32)
    if n:
        k = int(round(nan_frac * n))
        idx = rng.permutation(n)
        pts[idx[:k], rng.integers(3, size=k)] = np.nan
        j = int(round(inf_frac * n))
        pts[idx[k:k + j], rng.integers(3, size=j)] = np.where(rng.uniform(size=j) < 0.5,
                                                               np.inf, -np.inf)
    return pts


def sensor_poses(n_frames: int, seed: int = 2, *, band=(0.05, 2.0)):
    """Camera-to-map poses, float32 [F, 3, 4] row-major [R|t], and height bands [F, 2].

    The camera's optical frame (x right, y down, z forward) is mounted level on a robot
    at a random heading: map = Rz(yaw) @ M @ optical + t, with M taking forward to map x,
    right to map -y and down to map -z; t = (x, y, h), x, y uniform in [0, 40] m and the
    lens height h uniform in [0.8, 1.2] m.  Every frame keeps heights ``band`` (metres
    above the floor, in the map frame)."""
    rng = _rng(seed)
    M = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])
    out = np.zeros((n_frames, 3, 4), np.float32)
    for f in range(n_frames):
        yaw = rng.uniform(0.0, 2.0 * np.pi)
        c, s_ = np.cos(yaw), np.sin(yaw)
        rz = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])
        out[f, :, :3] = rz @ M
        out[f, :, 3] = (rng.uniform(0, 40), rng.uniform(0, 40), rng.uniform(0.8, 1.2))
    bands = np.tile(np.asarray(band, np.float32), (n_frames, 1))
    return out, bands
