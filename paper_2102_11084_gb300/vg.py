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

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvg.so")
_LOCK = threading.Lock()
_LIB = None

ORIGIN_FROM_MIN = 1
METHOD_AUTO = 0
METHOD_SORT = 16
_METHODS = {"auto": METHOD_AUTO, "sort": METHOD_SORT}
MAX_POINTS = (1 << 30) - 1


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
                    method="sort", stream: Optional[torch.cuda.Stream] = None,
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


def downsample(xyz: torch.Tensor, leaf: float, origin: Optional[torch.Tensor] = None, *,
               method="sort", point_to_voxel: bool = False,
               stream: Optional[torch.cuda.Stream] = None) -> Decimation:
    """Voxel-grid decimation of one cloud: centroid per occupied voxel, key order.

    ``origin`` None means the per-axis minimum of the valid points.  Synchronises the
    stream once to read V and the device error word.
    """
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
                       method="sort", point_to_voxel: bool = False,
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


def set_spin_limit(limit: int) -> None:
    """Test hook: bound every chained-scan wait (0 = default)."""
    lib().vg_debug_set_spin_limit(int(limit))
