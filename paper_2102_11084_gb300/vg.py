"""Python binding of libvg.so (include/vg.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module checks tensors,
allocates outputs and workspace with PyTorch (device memory, streams), calls the C ABI
and trims the outputs.  There is no CPU fallback: if the library is missing or the
tensors are not on a CUDA device, the call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from enum import IntEnum
from typing import NamedTuple, Optional

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvg.so")
_LOCK = threading.Lock()
_LIB = None

ORIGIN_FROM_MIN = 1
METHOD_AUTO = 0
METHOD_SORT = 16
METHOD_HASH = 32
SORT_BUCKETS = 2
SORT_LSD = 4
USE_GRAPH = 64
SORT_FRAME = 128
GRID_SHIFT = 8
# "auto" (the default): "sort" for clouds of 4,194,304 points or more, else "sort_lsd";
# "sort": 32-bit keys grouped by buckets (partition passes over the top key bits, every
# bucket reduced on chip), otherwise a global radix sort; "sort_lsd": every key digit in a
# global radix pass and the segmented reduction; "sort_bucket": the same as "sort" (kept
# for compatibility); "frame": one camera frame counted into bins of 2^12 keys and reduced
# bin by bin (five kernels; 32-bit keys); "hash": hash-table accumulation.  All give
# identical rows.
_METHODS = {"auto": METHOD_AUTO, "sort": METHOD_SORT,
            "sort_bucket": METHOD_SORT | SORT_BUCKETS, "sort_lsd": METHOD_SORT | SORT_LSD,
            "frame": METHOD_SORT | SORT_FRAME, "hash": METHOD_HASH}
MAX_POINTS = (1 << 30) - 1
MAX_FRAMES = 1024
MAX_LEVELS = 8


class Status(IntEnum):
    OK = 0
    INVALID_ARG = 1
    ALIGN = 2
    RANGE = 3
    CAPACITY = 4
    WORKSPACE = 5
    TIMEOUT = 6
    CUDA = 7


class VGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {status_string(status)} (status {int(status)})")


_SIGS = {
    "vg_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "vg_version": ([], ctypes.c_int),
    "vg_downsample_workspace_bytes": ([ctypes.c_int64, ctypes.c_int], ctypes.c_size_t),
    "vg_frame_one_launch_points": ([ctypes.c_int], ctypes.c_int64),
    "vg_downsample": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_float,
                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                       ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "vg_debug_set_spin_limit": ([ctypes.c_uint32], None),
    "vg_downsample_noalloc": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_float,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                               ctypes.c_void_p], ctypes.c_int),
    "vg_downsample_noalloc_scratch_bytes": ([], ctypes.c_size_t),
    "vg_set_stage_events": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "vg_debug_grid_barrier_timeout": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                       ctypes.c_void_p], ctypes.c_int),
    "vg_debug_wait_timeout": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p],
                              ctypes.c_int),
    "vg_batch_workspace_bytes": ([ctypes.c_int64, ctypes.c_int, ctypes.c_int], ctypes.c_size_t),
    "vg_downsample_frames": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                              ctypes.c_void_p], ctypes.c_int),
    "vg_downsample_frames_posed": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "vg_downsample_ex_workspace_bytes": ([ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p], ctypes.c_size_t),
    "vg_downsample_frames_ex": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                 ctypes.c_void_p], ctypes.c_int),
    "vg_map_create": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_float],
                      ctypes.c_int),
    "vg_map_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "vg_map_clear": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "vg_map_insert": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                       ctypes.c_void_p], ctypes.c_int),
    "vg_map_extract": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                       ctypes.c_int),
    "vg_thin_workspace_bytes": ([ctypes.c_int64], ctypes.c_size_t),
    "vg_thin": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_float, ctypes.c_float,
                 ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                 ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "vg_plan_create": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int], ctypes.c_int),
    "vg_plan_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "vg_plan_configure": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "vg_plan_get": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                    ctypes.c_int),
    "vg_downsample_batch": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                             ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
                            ctypes.c_int),
    "vg_plan_tune": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                      ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                      ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                      ctypes.c_void_p], ctypes.c_int),
    "vg_pyramid_workspace_bytes": ([ctypes.c_int64, ctypes.c_int, ctypes.c_int], ctypes.c_size_t),
    "vg_pyramid": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_float, ctypes.c_int,
                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                    ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "vg_downsample_backward": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                               ctypes.c_int),
}


def lib():
    """The loaded libvg.so; raises if it has not been built."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libvg.so not found at {LIB_PATH}: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            h = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                fn = getattr(h, name)
                fn.argtypes = args
                fn.restype = res
            _LIB = h
    return _LIB


def status_string(status: int) -> str:
    return lib().vg_status_string(int(status)).decode()


def version() -> int:
    return int(lib().vg_version())


def _check(status: int, where: str):
    if status != 0:
        raise VGError(status, where)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _cuda_cloud(xyz: torch.Tensor) -> torch.Tensor:
    if not isinstance(xyz, torch.Tensor) or not xyz.is_cuda:
        raise TypeError("xyz must be a CUDA tensor (the library has no CPU path)")
    if xyz.dtype != torch.float32 or xyz.dim() != 2 or xyz.shape[1] != 3:
        raise TypeError("xyz must be float32 [N, 3]")
    if not xyz.is_contiguous():
        raise ValueError("xyz must be contiguous")
    if xyz.shape[0] > MAX_POINTS:
        raise ValueError(f"at most {MAX_POINTS} points per call")
    return xyz


def method_flag(method) -> int:
    if isinstance(method, int):
        return method
    return _METHODS[method]


def workspace_bytes(n: int, flags: int = 0) -> int:
    return int(lib().vg_downsample_workspace_bytes(int(n), int(flags)))


def frame_one_launch_points(posed: bool = False) -> int:
    """Largest frame method="frame" groups in one cooperative launch on this device (0: none)."""
    return int(lib().vg_frame_one_launch_points(1 if posed else 0))


class Buffers(NamedTuple):
    """Outputs and scratch of one decimation call (device tensors, capacity-sized)."""
    origin: torch.Tensor          # float32 [3]
    keys: torch.Tensor            # uint64 as int64 [cap]
    centroids: torch.Tensor       # float32 [cap, 3]
    counts: torch.Tensor          # uint32 as int32 [cap]
    num_voxels: torch.Tensor      # int64 [1]
    error: torch.Tensor           # int32 [1]
    point_to_voxel: Optional[torch.Tensor]  # int32 [N]
    workspace: torch.Tensor       # uint8


def alloc_buffers(n: int, device, *, cap: Optional[int] = None, point_to_voxel: bool = False,
                  flags: int = 0, origin: Optional[torch.Tensor] = None) -> Buffers:
    cap = n if cap is None else int(cap)
    dev = torch.device(device)
    o = torch.zeros(3, dtype=torch.float32, device=dev) if origin is None else origin
    return Buffers(
        origin=o,
        keys=torch.empty(max(cap, 1), dtype=torch.int64, device=dev),
        centroids=torch.empty((max(cap, 1), 3), dtype=torch.float32, device=dev),
        counts=torch.empty(max(cap, 1), dtype=torch.int32, device=dev),
        num_voxels=torch.zeros(1, dtype=torch.int64, device=dev),
        error=torch.zeros(1, dtype=torch.int32, device=dev),
        point_to_voxel=(torch.empty(max(n, 1), dtype=torch.int32, device=dev)
                        if point_to_voxel else None),
        workspace=torch.empty(max(workspace_bytes(n, flags), 256), dtype=torch.uint8, device=dev),
    )


def downsample_into(xyz: torch.Tensor, leaf: float, buf: Buffers, *, origin_from_min: bool,
                    method="auto", stream: Optional[torch.cuda.Stream] = None,
                    cap: Optional[int] = None) -> None:
    """Launch vg_downsample into preallocated buffers (asynchronous, no host sync)."""
    xyz = _cuda_cloud(xyz)
    n = xyz.shape[0]
    flags = method_flag(method) | (ORIGIN_FROM_MIN if origin_from_min else 0)
    cap = buf.keys.shape[0] if cap is None else cap
    st = lib().vg_downsample(
        _ptr(xyz), n, _ptr(buf.origin), ctypes.c_float(leaf), _ptr(buf.keys), _ptr(buf.centroids),
        _ptr(buf.counts), int(cap), _ptr(buf.num_voxels), _ptr(buf.point_to_voxel),
        _ptr(buf.error), _ptr(buf.workspace), buf.workspace.numel(), flags, _stream_ptr(stream))
    _check(st, "vg_downsample")


class Decimation(NamedTuple):
    keys: torch.Tensor            # int64 view of the uint64 keys [V], ascending as unsigned
    centroids: torch.Tensor       # float32 [V, 3]
    counts: torch.Tensor          # int32 [V]
    origin: torch.Tensor          # float32 [3]
    point_to_voxel: Optional[torch.Tensor]  # int32 [N], -1 = invalid point
    attrs: Optional[torch.Tensor] = None    # float32 [V, C] per-voxel attribute means


def downsample(xyz: torch.Tensor, leaf: float, origin: Optional[torch.Tensor] = None, *,
               method="auto", point_to_voxel: bool = False, pose=None, z_limits=None,
               attrs=None, min_count: int = 1,
               stream: Optional[torch.cuda.Stream] = None) -> Decimation:
    """Voxel-grid decimation of one cloud: centroid per occupied voxel, key order.

    ``origin`` None means the per-axis minimum of the valid points.  ``pose`` ([3,4]
    [R|t]) and ``z_limits`` ([z_min, z_max]) first take the cloud into the common frame
    and drop points outside the height band; ``attrs`` (uint8 [N, C], C <= 4) adds
    per-voxel attribute means and ``min_count`` removes voxels with fewer points
    (vg_downsample_frames_ex).  Synchronises the stream once to read V and the device
    error word.
    """
    if pose is not None or z_limits is not None or attrs is not None or min_count > 1:
        fr = downsample_frames([xyz], [leaf], None if origin is None else [origin],
                               method=method, point_to_voxel=point_to_voxel,
                               poses=None if pose is None else [pose],
                               z_limits=None if z_limits is None else [z_limits],
                               attrs=None if attrs is None else [attrs], min_count=min_count,
                               stream=stream)
        return Decimation(fr.keys, fr.centroids, fr.counts, fr.origins[0], fr.point_to_voxel,
                          fr.attrs)
    xyz = _cuda_cloud(xyz)
    n = xyz.shape[0]
    org = None
    if origin is not None:
        org = torch.as_tensor(origin, dtype=torch.float32, device=xyz.device).reshape(3).contiguous()
    buf = alloc_buffers(n, xyz.device, point_to_voxel=point_to_voxel,
                        flags=method_flag(method), origin=org)
    downsample_into(xyz, leaf, buf, origin_from_min=origin is None, method=method, stream=stream,
                    cap=n)
    (stream or torch.cuda.current_stream()).synchronize()
    err = int(buf.error.item())
    _check(err, "vg_downsample (device)")
    v = int(buf.num_voxels.item())
    return Decimation(buf.keys[:v], buf.centroids[:v], buf.counts[:v], buf.origin,
                      buf.point_to_voxel[:n] if point_to_voxel else None)


NOALLOC_MAX_POINTS = 1 << 20


def downsample_noalloc(xyz: torch.Tensor, leaf: float, origin: Optional[torch.Tensor] = None, *,
                       method="auto", point_to_voxel: bool = False,
                       stream: Optional[torch.cuda.Stream] = None) -> Decimation:
    """vg_downsample_noalloc: decimation whose scratch is the library's static device
    array instead of a workspace (for callers that cannot allocate device memory; the
    outputs here are still torch tensors).  At most NOALLOC_MAX_POINTS points; calls
    that overlap on the GPU race on the shared scratch."""
    xyz = _cuda_cloud(xyz)
    n = xyz.shape[0]
    dev = xyz.device
    org = (torch.zeros(3, dtype=torch.float32, device=dev) if origin is None else
           torch.as_tensor(origin, dtype=torch.float32, device=dev).reshape(3).contiguous())
    cap = max(n, 1)
    keys = torch.empty(cap, dtype=torch.int64, device=dev)
    cents = torch.empty((cap, 3), dtype=torch.float32, device=dev)
    counts = torch.empty(cap, dtype=torch.int32, device=dev)
    nv = torch.zeros(1, dtype=torch.int64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    p2v = torch.empty(cap, dtype=torch.int32, device=dev) if point_to_voxel else None
    flags = method_flag(method) | (ORIGIN_FROM_MIN if origin is None else 0)
    st = lib().vg_downsample_noalloc(
        _ptr(xyz), n, _ptr(org), ctypes.c_float(leaf), _ptr(keys), _ptr(cents), _ptr(counts), n,
        _ptr(nv), _ptr(p2v), _ptr(err), flags, _stream_ptr(stream))
    _check(st, "vg_downsample_noalloc")
    (stream or torch.cuda.current_stream()).synchronize()
    _check(int(err.item()), "vg_downsample_noalloc (device)")
    v = int(nv.item())
    return Decimation(keys[:v], cents[:v], counts[:v], org, p2v[:n] if point_to_voxel else None)


# ---- batched frames (step a8) -------------------------------------------------------
class Frames(NamedTuple):
    """Outputs of a batched call: frame f's voxels are rows offsets[f]:offsets[f+1]."""
    keys: torch.Tensor            # int64 view of uint64 per-frame keys [V_total]
    centroids: torch.Tensor       # float32 [V_total, 3]
    counts: torch.Tensor          # int32 [V_total]
    offsets: list                 # host list of F+1 row offsets
    origins: torch.Tensor         # float32 [F, 3]
    point_to_voxel: Optional[torch.Tensor]  # int32 [N_total], global rows
    attrs: Optional[torch.Tensor] = None    # float32 [V_total, C] per-voxel attribute means

    def frame(self, f: int) -> Decimation:
        a, b = self.offsets[f], self.offsets[f + 1]
        return Decimation(self.keys[a:b], self.centroids[a:b], self.counts[a:b], self.origins[f],
                          None, None if self.attrs is None else self.attrs[a:b])


class VoxelExtras(ctypes.Structure):
    """vg_voxel_extras of include/vg.h."""
    _fields_ = [("attrs", ctypes.c_void_p), ("attr_channels", ctypes.c_int),
                ("out_attrs", ctypes.c_void_p), ("min_count", ctypes.c_uint32)]


def _is_cat_form(frames) -> bool:
    """True for the (xyz [N,3], offsets [F+1]) form, False for a list of clouds."""
    return (isinstance(frames, tuple) and len(frames) == 2 and isinstance(frames[0], torch.Tensor)
            and not (isinstance(frames[1], torch.Tensor) and frames[1].dim() == 2))


def _frame_inputs(frames, leaves, origins, device):
    """Concatenate a list of [N_f,3] clouds (or take (xyz, offsets) as given)."""
    if not _is_cat_form(frames):
        sizes = [int(f.shape[0]) for f in frames]
        xyz = torch.cat([f.to(device=device, dtype=torch.float32) for f in frames]).contiguous() \
            if frames else torch.zeros((0, 3), dtype=torch.float32, device=device)
        offs = [0]
        for n in sizes:
            offs.append(offs[-1] + n)
    else:
        xyz, offs = frames
        offs = [int(v) for v in offs]
    F = len(offs) - 1
    off_t = torch.tensor(offs, dtype=torch.int64, device=device)
    lv = torch.as_tensor(leaves, dtype=torch.float32).reshape(F).to(device)
    og = (torch.zeros((F, 3), dtype=torch.float32, device=device) if origins is None else
          _per_frame(origins, F, 3, device))
    return _cuda_cloud(xyz), off_t, F, lv, og


def _per_frame(values, F: int, width: int, device) -> Optional[torch.Tensor]:
    if values is None:
        return None
    if isinstance(values, (list, tuple)) and values and isinstance(values[0], torch.Tensor):
        values = torch.stack([v.to(device=device, dtype=torch.float32).reshape(-1)
                              for v in values])
    elif not isinstance(values, torch.Tensor):
        values = np.asarray([np.asarray(v, np.float32) for v in values], np.float32)
    return torch.as_tensor(values, dtype=torch.float32).reshape(F, width).to(device).contiguous()


def downsample_frames(frames, leaves, origins=None, *, method="auto", point_to_voxel=False,
                      grid_per_sm: int = 0, poses=None, z_limits=None, attrs=None,
                      min_count: int = 1,
                      stream: Optional[torch.cuda.Stream] = None) -> Frames:
    """vg_downsample_frames: every frame decimated as it would be alone, in one call.

    ``frames`` is a list of float32 [N_f, 3] CUDA tensors or a tuple (xyz [N,3], offsets).
    ``origins`` None means each frame's minimum.  ``poses`` ([F,3,4] sensor poses [R|t])
    and ``z_limits`` ([F,2]) take each frame into the common frame and cut its height;
    ``attrs`` (uint8 [N_f, C] per frame, or [N, C] with the tuple form, C <= 4) gives
    per-voxel attribute means; ``min_count`` removes voxels with fewer points
    (vg_downsample_frames_ex).  Synchronises once to read the offsets.
    """
    dev = frames[0].device if len(frames) else torch.device("cuda")
    xyz, off_t, F, lv, og = _frame_inputs(frames, leaves, origins, dev)
    pz = _per_frame(poses, F, 12, dev)
    zl = _per_frame(z_limits, F, 2, dev)
    at = None
    if attrs is not None:
        at = attrs if isinstance(attrs, torch.Tensor) else torch.cat(
            [torch.as_tensor(a).reshape(int(f.shape[0]), -1) for a, f in zip(attrs, frames)])
        at = at.to(device=dev, dtype=torch.uint8).contiguous()
        if at.dim() != 2 or at.shape[0] != xyz.shape[0] or not 1 <= at.shape[1] <= 4:
            raise ValueError("attrs must be uint8 [N, C] with 1 <= C <= 4")
    n = xyz.shape[0]
    flags = method_flag(method) | (ORIGIN_FROM_MIN if origins is None else 0) | \
        (int(grid_per_sm) << GRID_SHIFT)
    cap = max(n, 1)
    keys = torch.empty(cap, dtype=torch.int64, device=dev)
    cents = torch.empty((cap, 3), dtype=torch.float32, device=dev)
    counts = torch.empty(cap, dtype=torch.int32, device=dev)
    out_off = torch.zeros(F + 1, dtype=torch.int64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    p2v = torch.empty(cap, dtype=torch.int32, device=dev) if point_to_voxel else None
    out_at = (torch.empty((cap, at.shape[1]), dtype=torch.float32, device=dev)
              if at is not None else None)
    ex = None
    if at is not None or min_count > 1:
        ex = VoxelExtras(None if at is None else at.data_ptr(), 0 if at is None else at.shape[1],
                         None if out_at is None else out_at.data_ptr(), int(min_count))
    wsb = (lib().vg_downsample_ex_workspace_bytes(n, F, flags, ctypes.byref(ex)) if ex else
           lib().vg_batch_workspace_bytes(n, F, flags))
    ws = torch.empty(max(int(wsb), 256), dtype=torch.uint8, device=dev)
    if pz is None and zl is None and ex is None:
        st = lib().vg_downsample_frames(
            _ptr(xyz), n, _ptr(off_t), F, _ptr(og), _ptr(lv), _ptr(keys), _ptr(cents),
            _ptr(counts), n, _ptr(out_off), _ptr(p2v), _ptr(err), _ptr(ws), ws.numel(), flags,
            _stream_ptr(stream))
    else:
        st = lib().vg_downsample_frames_ex(
            _ptr(xyz), n, _ptr(off_t), F, _ptr(pz), _ptr(zl), _ptr(og), _ptr(lv), _ptr(keys),
            _ptr(cents), _ptr(counts), n, _ptr(out_off), _ptr(p2v),
            ctypes.byref(ex) if ex else None, _ptr(err), _ptr(ws), ws.numel(), flags,
            _stream_ptr(stream))
    _check(st, "vg_downsample_frames")
    (stream or torch.cuda.current_stream()).synchronize()
    _check(int(err.item()), "vg_downsample_frames (device)")
    offs = out_off.cpu().tolist()
    v = offs[-1]
    return Frames(keys[:v], cents[:v], counts[:v], offs, og, p2v[:n] if point_to_voxel else None,
                  None if out_at is None else out_at[:v])


def frames_into(xyz: torch.Tensor, frame_offsets: torch.Tensor, n_frames: int,
                origins: torch.Tensor, leaves: torch.Tensor, out_keys: torch.Tensor,
                out_centroids: torch.Tensor, out_counts: torch.Tensor,
                out_frame_offsets: torch.Tensor, out_error: torch.Tensor,
                workspace: torch.Tensor, *, origin_from_min: bool = True, method="auto",
                poses: Optional[torch.Tensor] = None, z_limits: Optional[torch.Tensor] = None,
                point_to_voxel: Optional[torch.Tensor] = None,
                attrs: Optional[torch.Tensor] = None, out_attrs: Optional[torch.Tensor] = None,
                min_count: int = 1, stream: Optional[torch.cuda.Stream] = None) -> None:
    """Launch vg_downsample_frames (or _ex, when poses, z_limits, attrs or min_count are
    given) into preallocated device buffers; asynchronous, no host sync.  The workspace
    must hold ex_workspace_bytes(...) for attrs/min_count."""
    xyz = _cuda_cloud(xyz)
    flags = method_flag(method) | (ORIGIN_FROM_MIN if origin_from_min else 0)
    head = (_ptr(origins), _ptr(leaves), _ptr(out_keys), _ptr(out_centroids), _ptr(out_counts),
            out_keys.shape[0], _ptr(out_frame_offsets), _ptr(point_to_voxel))
    tail = (_ptr(out_error), _ptr(workspace), workspace.numel(), flags, _stream_ptr(stream))
    ex = extras(attrs, out_attrs, min_count)
    if poses is None and z_limits is None and ex is None:
        st = lib().vg_downsample_frames(_ptr(xyz), xyz.shape[0], _ptr(frame_offsets),
                                        int(n_frames), *head, *tail)
    else:
        st = lib().vg_downsample_frames_ex(_ptr(xyz), xyz.shape[0], _ptr(frame_offsets),
                                           int(n_frames), _ptr(poses), _ptr(z_limits), *head,
                                           ctypes.byref(ex) if ex else None, *tail)
    _check(st, "vg_downsample_frames")


def extras(attrs: Optional[torch.Tensor] = None, out_attrs: Optional[torch.Tensor] = None,
           min_count: int = 1) -> Optional[VoxelExtras]:
    """The vg_voxel_extras of a call, or None when it asks for nothing extra."""
    if attrs is None and min_count <= 1:
        return None
    return VoxelExtras(None if attrs is None else attrs.data_ptr(),
                       0 if attrs is None else int(attrs.shape[1]),
                       None if out_attrs is None else out_attrs.data_ptr(), int(min_count))


def ex_workspace_bytes(n_total: int, n_frames: int, flags: int, ex: Optional[VoxelExtras]) -> int:
    return int(lib().vg_downsample_ex_workspace_bytes(
        int(n_total), int(n_frames), int(flags), ctypes.byref(ex) if ex else None))


class Thinned(NamedTuple):
    keep: torch.Tensor            # bool [N]: the points that remain
    num_kept: int
    passes: int                   # passes of the loop
    origin: torch.Tensor          # float32 [3]


def thin(xyz: torch.Tensor, cell: float, threshold: int, priority: torch.Tensor, *,
         radius: Optional[float] = None, batch: int = 1000,
         origin: Optional[torch.Tensor] = None,
         stream: Optional[torch.cuda.Stream] = None) -> Thinned:
    """vg_thin: the paper's neighbour-count thinning loop (radius defaults to the cell
    edge; ``priority`` uint32 [N] on the device orders the deleted batches)."""
    xyz = _cuda_cloud(xyz)
    n = xyz.shape[0]
    dev = xyz.device
    pr = priority.to(device=dev, dtype=torch.int32).contiguous() if priority.dtype != torch.int32 \
        else priority.contiguous()
    if pr.numel() != n:
        raise ValueError("priority must have one entry per point")
    org = (torch.zeros(3, dtype=torch.float32, device=dev) if origin is None else
           torch.as_tensor(origin, dtype=torch.float32, device=dev).reshape(3).contiguous())
    keep = torch.zeros(max(n, 1), dtype=torch.uint8, device=dev)
    kept = torch.zeros(1, dtype=torch.int64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(max(int(lib().vg_thin_workspace_bytes(n)), 256), dtype=torch.uint8,
                     device=dev)
    passes = ctypes.c_int32(0)
    st = lib().vg_thin(_ptr(xyz), n, _ptr(org), ctypes.c_float(cell),
                       ctypes.c_float(cell if radius is None else radius), int(threshold),
                       int(batch), _ptr(pr), _ptr(keep), _ptr(kept), ctypes.byref(passes),
                       _ptr(err), _ptr(ws), ws.numel(), ORIGIN_FROM_MIN if origin is None else 0,
                       _stream_ptr(stream))
    _check(st, "vg_thin")
    (stream or torch.cuda.current_stream()).synchronize()
    _check(int(err.item()), "vg_thin (device)")
    return Thinned(keep[:n].bool(), int(kept.item()), int(passes.value), org)


class VoxelMap:
    """vg_map: a device-resident voxel map on one fixed lattice (origin, leaf) that frames
    are merged into.  Extracting gives what one decimation of every inserted point with
    that origin would give."""

    def __init__(self, capacity: int, origin, leaf: float, device="cuda"):
        self.device = torch.device(device)
        self.origin = np.ascontiguousarray(np.asarray(origin, np.float32).reshape(3))
        self.leaf = float(leaf)
        self.capacity = int(capacity)
        self.error = torch.zeros(1, dtype=torch.int32, device=self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().vg_map_create(ctypes.byref(h), self.capacity,
                                       self.origin.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.c_float(self.leaf)), "vg_map_create")
        self._h = h

    def insert(self, frames, poses=None, z_limits=None,
               stream: Optional[torch.cuda.Stream] = None) -> None:
        """Adds the valid points of one cloud ([N,3] CUDA tensor), a list of clouds or an
        (xyz, offsets) tuple; asynchronous."""
        if isinstance(frames, torch.Tensor):
            frames = [frames]
        xyz, off_t, F, _, _ = _frame_inputs(frames, [self.leaf] * (
            len(frames) if not _is_cat_form(frames) else len(frames[1]) - 1), None, self.device)
        pz = _per_frame(poses, F, 12, self.device)
        zl = _per_frame(z_limits, F, 2, self.device)
        self._keep = (xyz, off_t, pz, zl)  # alive until the launch has read them
        _check(lib().vg_map_insert(self._h, _ptr(xyz), xyz.shape[0], _ptr(off_t), F, _ptr(pz),
                                   _ptr(zl), _ptr(self.error), _stream_ptr(stream)),
               "vg_map_insert")

    def extract(self, cap: Optional[int] = None,
                stream: Optional[torch.cuda.Stream] = None) -> Decimation:
        """Every voxel of the map in ascending key order (synchronises once)."""
        cap = self.capacity * 2 if cap is None else int(cap)
        d = self.device
        keys = torch.empty(max(cap, 1), dtype=torch.int64, device=d)
        cents = torch.empty((max(cap, 1), 3), dtype=torch.float32, device=d)
        counts = torch.empty(max(cap, 1), dtype=torch.int32, device=d)
        nv = torch.zeros(1, dtype=torch.int64, device=d)
        _check(lib().vg_map_extract(self._h, _ptr(keys), _ptr(cents), _ptr(counts), cap, _ptr(nv),
                                    _ptr(self.error), _stream_ptr(stream)), "vg_map_extract")
        (stream or torch.cuda.current_stream(d)).synchronize()
        _check(int(self.error.item()), "vg_map (device)")
        v = int(nv.item())
        return Decimation(keys[:v], cents[:v], counts[:v],
                          torch.from_numpy(self.origin.copy()).to(d), None)

    def clear(self, stream: Optional[torch.cuda.Stream] = None) -> None:
        _check(lib().vg_map_clear(self._h, _stream_ptr(stream)), "vg_map_clear")
        self.error.zero_()

    def close(self) -> None:
        if getattr(self, "_h", None):
            torch.cuda.synchronize(self.device)
            lib().vg_map_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A batch plan (vg_plan): owned workspace, tuned method/grid, CUDA-graph replay."""

    def __init__(self, max_frames: int, max_points: int, method="auto"):
        h = ctypes.c_void_p()
        _check(lib().vg_plan_create(ctypes.byref(h), int(max_frames), int(max_points),
                                    method_flag(method)), "vg_plan_create")
        self._h = h
        self.max_frames = int(max_frames)
        self.max_points = int(max_points)

    def close(self):
        if getattr(self, "_h", None):
            lib().vg_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, method, grid_per_sm: int = 0):
        _check(lib().vg_plan_configure(self._h, method_flag(method), int(grid_per_sm)),
               "vg_plan_configure")

    def get(self):
        m, g, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check(lib().vg_plan_get(self._h, ctypes.byref(m), ctypes.byref(g), ctypes.byref(w)),
               "vg_plan_get")
        return {"method": {METHOD_AUTO: "auto", METHOD_SORT: "sort",
                           METHOD_SORT | SORT_LSD: "sort_lsd",
                           METHOD_SORT | SORT_FRAME: "frame", METHOD_HASH: "hash"}[m.value],
                "grid_per_sm": g.value, "workspace_bytes": w.value}

    def run(self, xyz, frame_offsets, n_frames, origins, leaves, out_keys, out_centroids,
            out_counts, out_frame_offsets, out_error, *, origin_from_min=True, graph=True,
            point_to_voxel=None, stream: Optional[torch.cuda.Stream] = None):
        """vg_downsample_batch into preallocated device tensors (no host sync)."""
        flags = (ORIGIN_FROM_MIN if origin_from_min else 0) | (USE_GRAPH if graph else 0)
        st = lib().vg_downsample_batch(
            self._h, _ptr(xyz), xyz.shape[0], _ptr(frame_offsets), int(n_frames), _ptr(origins),
            _ptr(leaves), _ptr(out_keys), _ptr(out_centroids), _ptr(out_counts),
            out_keys.shape[0], _ptr(out_frame_offsets), _ptr(point_to_voxel), _ptr(out_error),
            flags, _stream_ptr(stream))
        _check(st, "vg_downsample_batch")

    def tune(self, xyz, frame_offsets, n_frames, origins, leaves, out_keys, out_centroids,
             out_counts, out_frame_offsets, out_error, *, origin_from_min=True, reps=5,
             stream: Optional[torch.cuda.Stream] = None):
        """vg_plan_tune: time sort/sort_lsd/frame/hash x grids {4,8,16}; keeps the fastest
        (-1: not timed, or the grouping recorded a device error)."""
        ms = (ctypes.c_float * 12)()
        flags = ORIGIN_FROM_MIN if origin_from_min else 0
        st = lib().vg_plan_tune(
            self._h, _ptr(xyz), xyz.shape[0], _ptr(frame_offsets), int(n_frames), _ptr(origins),
            _ptr(leaves), _ptr(out_keys), _ptr(out_centroids), _ptr(out_counts),
            out_keys.shape[0], _ptr(out_frame_offsets), _ptr(out_error), flags, int(reps),
            _stream_ptr(stream), ms)
        _check(st, "vg_plan_tune")
        names = [f"{m}@{g}" for m in ("sort", "sort_lsd", "frame", "hash") for g in (4, 8, 16)]
        self.last_tuning = dict(zip(names, list(ms)))
        return self.last_tuning

    def save_tuning(self, path: str, workload: str = "") -> None:
        """Writes the plan's chosen method and grid (and the timings that chose them) to a
        JSON file, so that a later process can skip the tuning runs."""
        import json
        rec = {"max_frames": self.max_frames, "max_points": self.max_points,
               "workload": workload, "device": torch.cuda.get_device_name(),
               **{k: v for k, v in self.get().items() if k != "workspace_bytes"},
               "candidates_ms": getattr(self, "last_tuning", None)}
        with open(path, "w") as f:
            json.dump(rec, f, indent=1)

    def load_tuning(self, path: str) -> dict:
        """Applies a choice written by save_tuning (same plan sizes required)."""
        import json
        with open(path) as f:
            rec = json.load(f)
        if rec.get("max_frames") != self.max_frames or rec.get("max_points") != self.max_points:
            raise ValueError("tuning was recorded for a plan of other sizes")
        self.configure(rec["method"], int(rec["grid_per_sm"]))
        return rec


# ---- pyramid (step a6) -----------------------------------------------------------------
def pyramid(xyz: torch.Tensor, leaf: float, levels: int, origin: Optional[torch.Tensor] = None,
            *, point_to_voxel: bool = False, method="auto",
            stream: Optional[torch.cuda.Stream] = None) -> list:
    """vg_pyramid: level 0 = decimation at ``leaf``, level k+1 = merge of level k by key>>3.

    ``method``: "auto", "sort", "sort_lsd" or "sort_bucket" (level 0's grouping; "hash"
    is refused).  Returns a list of ``levels`` Decimation tuples (point_to_voxel only on
    level 0).
    """
    xyz = _cuda_cloud(xyz)
    n = xyz.shape[0]
    dev = xyz.device
    org = (torch.zeros(3, dtype=torch.float32, device=dev) if origin is None else
           torch.as_tensor(origin, dtype=torch.float32, device=dev).reshape(3).contiguous())
    cap = max(n * levels, 1)
    keys = torch.empty(cap, dtype=torch.int64, device=dev)
    cents = torch.empty((cap, 3), dtype=torch.float32, device=dev)
    counts = torch.empty(cap, dtype=torch.int32, device=dev)
    loff = torch.zeros(levels + 1, dtype=torch.int64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    p2v = torch.empty(max(n, 1), dtype=torch.int32, device=dev) if point_to_voxel else None
    if method_flag(method) & ~(METHOD_SORT | SORT_BUCKETS | SORT_LSD):  # (auto = 0 passes)
        raise ValueError("vg_pyramid groups level 0 by sorting")
    flags = (ORIGIN_FROM_MIN if origin is None else 0) | (method_flag(method) &
                                                          (SORT_BUCKETS | SORT_LSD))
    ws = torch.empty(max(int(lib().vg_pyramid_workspace_bytes(n, levels, flags)), 256),
                     dtype=torch.uint8, device=dev)
    st = lib().vg_pyramid(_ptr(xyz), n, _ptr(org), ctypes.c_float(leaf), int(levels), _ptr(keys),
                          _ptr(cents), _ptr(counts), cap, _ptr(loff), _ptr(p2v), _ptr(err),
                          _ptr(ws), ws.numel(), flags, _stream_ptr(stream))
    _check(st, "vg_pyramid")
    (stream or torch.cuda.current_stream()).synchronize()
    _check(int(err.item()), "vg_pyramid (device)")
    o = loff.cpu().tolist()
    out = []
    for k in range(levels):
        a, b = o[k], o[k + 1]
        out.append(Decimation(keys[a:b], cents[a:b], counts[a:b], org,
                              p2v[:n] if (point_to_voxel and k == 0) else None))
    return out


# ---- backward (step a7) ----------------------------------------------------------------
def backward(grad_centroids: torch.Tensor, counts: torch.Tensor, point_to_voxel: torch.Tensor,
             *, stream: Optional[torch.cuda.Stream] = None, check: bool = True) -> torch.Tensor:
    """vg_downsample_backward: grad_xyz[i] = grad_c[v(i)] / count[v(i)], 0 if invalid."""
    g = grad_centroids.contiguous().to(torch.float32)
    v = g.shape[0]
    n = point_to_voxel.shape[0]
    out = torch.empty((n, 3), dtype=torch.float32, device=g.device)
    err = torch.zeros(1, dtype=torch.int32, device=g.device)
    st = lib().vg_downsample_backward(_ptr(g), _ptr(counts.contiguous()),
                                      _ptr(point_to_voxel.contiguous()), n, v, _ptr(out), _ptr(err),
                                      _stream_ptr(stream))
    _check(st, "vg_downsample_backward")
    if check:
        (stream or torch.cuda.current_stream()).synchronize()
        _check(int(err.item()), "vg_downsample_backward (device)")
    return out


class VoxelDownsample(torch.autograd.Function):
    """centroids = VoxelDownsample.apply(xyz, leaf, origin): differentiable in xyz.

    Forward is vg_downsample (with point_to_voxel); backward is vg_downsample_backward.
    Keys and counts are returned as non-differentiable outputs.
    """

    @staticmethod
    def forward(ctx, xyz, leaf, origin=None):
        r = downsample(xyz.detach(), float(leaf), origin, point_to_voxel=True)
        ctx.save_for_backward(r.counts, r.point_to_voxel)
        ctx.mark_non_differentiable(r.keys, r.counts)
        return r.centroids, r.keys, r.counts

    @staticmethod
    def backward(ctx, grad_c, grad_keys=None, grad_counts=None):
        counts, p2v = ctx.saved_tensors
        if grad_c is None:
            return None, None, None
        return backward(grad_c, counts, p2v), None, None


def set_spin_limit(limit: int) -> None:
    """Test hook: bound every chained-scan wait (0 = default)."""
    lib().vg_debug_set_spin_limit(int(limit))
