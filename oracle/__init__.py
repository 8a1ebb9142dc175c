"""TEST INFRASTRUCTURE ONLY: the CPU oracle of voxel-grid decimation.

A plain, slow, FP64 restatement (``vg_oracle.cpp``, a ``std::map`` over voxel
triples) of what the GPU library computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.  It
shares no code with the CUDA sources and never imports the product package.

Functions follow arXiv 2102.11084 Sec. II-C (ordered subdivision of space, cell
table sorted by cell, one output point per occupied cell) with the voxel-grid
centroid definition of the PCL filter the paper replaces (Sec. I); the readings
where the paper is silent are listed at the top of ``vg_oracle.cpp``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import NamedTuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vg_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "libvg_oracle.so")
_LOCK = threading.Lock()
_LIB = None

STATUS_OK = 0
STATUS_RANGE = 3
STATUS_CAPACITY = 4


def build(force: bool = False) -> str:
    """Compile the oracle with strict IEEE binary32 semantics (no contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call([
        "g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
        "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            p = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.oracle_origin.argtypes = [p, i64, p]
            lib.oracle_origin.restype = i64
            lib.oracle_keys.argtypes = [p, i64, p, ctypes.c_float, p, p, p]
            lib.oracle_keys.restype = ctypes.c_int
            lib.oracle_downsample.argtypes = [p, i64, p, ctypes.c_float, p, p, p, i64, p, p]
            lib.oracle_downsample.restype = i64
            lib.oracle_pyramid_merge.argtypes = [p, p, p, i64, p, p, p]
            lib.oracle_pyramid_merge.restype = i64
            lib.oracle_backward.argtypes = [p, p, p, i64, p]
            lib.oracle_backward.restype = None
            lib.oracle_centroid_loss.argtypes = [p, i64, p, i64, p]
            lib.oracle_centroid_loss.restype = ctypes.c_double
            lib.oracle_pose.argtypes = [p, i64, p, p, p]
            lib.oracle_pose.restype = None
            lib.oracle_voxel_attrs.argtypes = [p, i64, p, ctypes.c_int, i64, p]
            lib.oracle_voxel_attrs.restype = None
            lib.oracle_min_count.argtypes = [p, p, p, p, ctypes.c_int, i64, ctypes.c_uint64, p,
                                             i64]
            lib.oracle_min_count.restype = i64
            lib.oracle_neighbor_counts.argtypes = [p, i64, p, p, ctypes.c_float, p]
            lib.oracle_neighbor_counts.restype = None
            lib.oracle_thin.argtypes = [p, i64, p, ctypes.c_float, ctypes.c_float, i64, i64, p, p]
            lib.oracle_thin.restype = i64
            _LIB = lib
    return _LIB


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _cloud(xyz) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32).reshape(-1, 3))
    return a


class Decimation(NamedTuple):
    keys: np.ndarray          # uint64 [V], ascending
    centroids: np.ndarray     # float64 [V, 3]
    counts: np.ndarray        # uint64 [V]
    point_to_voxel: np.ndarray  # int32 [N], -1 for invalid points
    origin: np.ndarray        # float32 [3]
    status: int


def origin(xyz) -> tuple[np.ndarray, int]:
    """Step a1: per-axis min over valid points (zeros when none); also #valid."""
    a = _cloud(xyz)
    out = np.zeros(3, np.float32)
    nvalid = _lib().oracle_origin(_ptr(a), a.shape[0], _ptr(out))
    return out, int(nvalid)


def keys(xyz, origin_xyz, leaf: float):
    """Step a2: (keys uint64 [N], ijk int64 [N,3], valid bool [N], status)."""
    a = _cloud(xyz)
    o = np.ascontiguousarray(np.asarray(origin_xyz, np.float32).reshape(3))
    n = a.shape[0]
    k = np.zeros(n, np.uint64)
    ijk = np.zeros((n, 3), np.int64)
    valid = np.zeros(n, np.uint8)
    st = _lib().oracle_keys(_ptr(a), n, _ptr(o), ctypes.c_float(leaf), _ptr(k), _ptr(ijk),
                            _ptr(valid))
    return k, ijk, valid.astype(bool), int(st)


def downsample(xyz, leaf: float, origin_xyz=None, cap: int | None = None) -> Decimation:
    """Steps a1-a5: centroid per occupied voxel in ascending Morton key order.

    ``origin_xyz`` None means the cloud minimum (step a1).
    """
    a = _cloud(xyz)
    n = a.shape[0]
    if origin_xyz is None:
        o, _ = origin(a)
    else:
        o = np.ascontiguousarray(np.asarray(origin_xyz, np.float32).reshape(3))
    cap = n if cap is None else int(cap)
    k = np.zeros(max(cap, 1), np.uint64)
    c = np.zeros((max(cap, 1), 3), np.float64)
    cnt = np.zeros(max(cap, 1), np.uint64)
    p2v = np.full(n, -1, np.int32)
    st = ctypes.c_int(0)
    v = _lib().oracle_downsample(_ptr(a), n, _ptr(o), ctypes.c_float(leaf), _ptr(k), _ptr(c),
                                 _ptr(cnt), cap, _ptr(p2v), ctypes.byref(st))
    m = min(int(v), cap)
    return Decimation(k[:m].copy(), c[:m].copy(), cnt[:m].copy(), p2v, o, int(st.value))


def pyramid_merge(keys_k, centroids_k, counts_k):
    """Step a6: merge one level by key >> 3, count-weighted, FP64."""
    kk = np.ascontiguousarray(keys_k, np.uint64)
    cc = np.ascontiguousarray(centroids_k, np.float64).reshape(-1, 3)
    nn = np.ascontiguousarray(counts_k, np.uint64)
    v = kk.shape[0]
    ok = np.zeros(max(v, 1), np.uint64)
    oc = np.zeros((max(v, 1), 3), np.float64)
    on = np.zeros(max(v, 1), np.uint64)
    m = _lib().oracle_pyramid_merge(_ptr(kk), _ptr(cc), _ptr(nn), v, _ptr(ok), _ptr(oc), _ptr(on))
    return ok[:m].copy(), oc[:m].copy(), on[:m].copy()


def pyramid(xyz, leaf: float, levels: int, origin_xyz=None):
    """Level 0 = decimation at ``leaf``; level k+1 = pyramid_merge(level k)."""
    d = downsample(xyz, leaf, origin_xyz)
    out = [(d.keys, d.centroids, d.counts)]
    for _ in range(1, levels):
        out.append(pyramid_merge(*out[-1]))
    return out, d


def backward(grad_centroids, counts, point_to_voxel) -> np.ndarray:
    """Step a7: grad_xyz[i] = grad_c[v(i)] / n[v(i)], 0 for invalid points (FP64)."""
    g = np.ascontiguousarray(grad_centroids, np.float64).reshape(-1, 3)
    nn = np.ascontiguousarray(counts, np.uint64)
    p2v = np.ascontiguousarray(point_to_voxel, np.int32)
    out = np.zeros((p2v.shape[0], 3), np.float64)
    _lib().oracle_backward(_ptr(g), _ptr(nn), _ptr(p2v), p2v.shape[0], _ptr(out))
    return out


def centroid_loss(xyz64, point_to_voxel, num_voxels: int, targets) -> float:
    """L = (1/(3V)) sum_v |c_v - t_v|^2 with FP64 coordinates and fixed membership."""
    x = np.ascontiguousarray(xyz64, np.float64).reshape(-1, 3)
    p2v = np.ascontiguousarray(point_to_voxel, np.int32)
    t = np.ascontiguousarray(targets, np.float64).reshape(-1, 3)
    return float(_lib().oracle_centroid_loss(_ptr(x), x.shape[0], _ptr(p2v), int(num_voxels),
                                             _ptr(t)))


def loss_grad_centroids(centroids, targets) -> np.ndarray:
    """dL/dc_v = 2 (c_v - t_v) / (3V) for the mean-squared centroid loss."""
    c = np.asarray(centroids, np.float64).reshape(-1, 3)
    t = np.asarray(targets, np.float64).reshape(-1, 3)
    v = c.shape[0]
    return 2.0 * (c - t) / (3.0 * v) if v else np.zeros((0, 3))


def downsample_batch(frames, leaves, origins=None):
    """Step a8 (the definition): every frame decimated on its own."""
    out = []
    for f, x in enumerate(frames):
        o = None if origins is None else origins[f]
        out.append(downsample(x, float(leaves[f]), o))
    return out


def pose(xyz, pose_rt=None, z_limits=None) -> np.ndarray:
    """Reading R12 (Sec. II-C: camera cloud into the global frame, height limit there):
    p' = R p + t per point in binary32, ((r0 x + r1 y) + r2 z) + t with one rounding per
    operation; points with p' not finite or z' outside [z_min, z_max] become NaN."""
    a = _cloud(xyz)
    out = np.empty_like(a)
    pr = None if pose_rt is None else np.ascontiguousarray(
        np.asarray(pose_rt, np.float32).reshape(12))
    zl = None if z_limits is None else np.ascontiguousarray(
        np.asarray(z_limits, np.float32).reshape(2))
    _lib().oracle_pose(_ptr(a), a.shape[0], None if pr is None else _ptr(pr),
                       None if zl is None else _ptr(zl), _ptr(out))
    return out


def downsample_posed(xyz, leaf: float, pose_rt=None, z_limits=None, origin_xyz=None):
    """A posed cloud decimated: the plain definition applied to pose(xyz)."""
    return downsample(pose(xyz, pose_rt, z_limits), leaf, origin_xyz)


class AttrDecimation(NamedTuple):
    keys: np.ndarray          # uint64 [V]
    centroids: np.ndarray     # float64 [V, 3]
    counts: np.ndarray        # uint64 [V]
    attrs: np.ndarray         # float32 [V, C] per-voxel channel means
    point_to_voxel: np.ndarray  # int32 [N]
    origin: np.ndarray        # float32 [3]


def downsample_attrs(xyz, leaf: float, attrs=None, min_count: int = 1, origin_xyz=None,
                     pose_rt=None, z_limits=None) -> AttrDecimation:
    """Readings R13/R14 on top of the (optionally posed) decimation: mean 8-bit
    attributes per voxel (exact sums, FP64 division, binary32 result) and removal of
    voxels with fewer than ``min_count`` points."""
    a = _cloud(xyz)
    d = downsample_posed(a, leaf, pose_rt, z_limits, origin_xyz) if (
        pose_rt is not None or z_limits is not None) else downsample(a, leaf, origin_xyz)
    n, v = a.shape[0], d.keys.shape[0]
    if attrs is None:
        at = np.zeros((n, 0), np.uint8)
    else:
        at = np.ascontiguousarray(np.asarray(attrs, np.uint8).reshape(n, -1))
    ch = at.shape[1]
    p2v = np.ascontiguousarray(d.point_to_voxel.astype(np.int32))
    out = np.zeros((max(v, 1), max(ch, 1)), np.float32)[:v, :ch].copy()
    if ch:
        _lib().oracle_voxel_attrs(_ptr(p2v), n, _ptr(at), ch, v, _ptr(out))
    keys = d.keys.copy()
    cents = np.ascontiguousarray(d.centroids.copy())
    counts = d.counts.copy()
    if min_count > 1 and v:
        out = np.ascontiguousarray(out)
        v = int(_lib().oracle_min_count(_ptr(keys), _ptr(cents), _ptr(counts),
                                        _ptr(out) if ch else None, ch, v, int(min_count),
                                        _ptr(p2v), n))
    return AttrDecimation(keys[:v], cents[:v], counts[:v], out[:v], p2v, d.origin)


def map_contents(frames, leaf: float, origin_xyz, poses=None, z_limits=None) -> Decimation:
    """A voxel map after inserting ``frames`` (each optionally posed and height-cut): by
    definition the decimation of all their points together on the map's lattice."""
    clouds = []
    for f, x in enumerate(frames):
        p = None if poses is None else poses[f]
        z = None if z_limits is None else z_limits[f]
        clouds.append(pose(x, p, z) if (p is not None or z is not None) else _cloud(x))
    allp = np.concatenate(clouds) if clouds else np.zeros((0, 3), np.float32)
    return downsample(allp, leaf, origin_xyz)


def neighbor_counts(xyz, ijk, alive, r: float) -> np.ndarray:
    """Reading R16, one count: for every remaining point, the other remaining points of
    the 27 surrounding cells within distance r (squared distance in binary32)."""
    a = _cloud(xyz)
    n = a.shape[0]
    ij = np.ascontiguousarray(np.asarray(ijk, np.int64).reshape(n, 3))
    al = np.ascontiguousarray(np.asarray(alive, np.uint8).reshape(n))
    out = np.zeros(max(n, 1), np.int64)
    _lib().oracle_neighbor_counts(_ptr(a), n, _ptr(ij), _ptr(al), ctypes.c_float(r), _ptr(out))
    return out[:n]


def thin(xyz, cell: float, threshold: int, priority, *, radius=None, batch: int = 1000,
         origin_xyz=None):
    """Reading R16: the paper's neighbour-count thinning loop (Algorithm 1) with the
    random choice of deleted points replaced by the lowest given priorities.  Returns
    (keep bool [N], passes of the loop, status)."""
    a = _cloud(xyz)
    n = a.shape[0]
    o = origin(a)[0] if origin_xyz is None else np.ascontiguousarray(
        np.asarray(origin_xyz, np.float32).reshape(3))
    pr = np.ascontiguousarray(np.asarray(priority, np.uint32).reshape(n))
    keep = np.zeros(max(n, 1), np.uint8)
    r = float(cell) if radius is None else float(radius)
    res = int(_lib().oracle_thin(_ptr(a), n, _ptr(o), ctypes.c_float(cell), ctypes.c_float(r),
                                 int(threshold), int(batch), _ptr(pr), _ptr(keep)))
    if res < 0:
        return keep[:n].astype(bool), 0, -res
    return keep[:n].astype(bool), res, STATUS_OK
