"""vg_downsample_noalloc (the entry point for callers that cannot allocate device
memory) must give what vg_downsample gives, call after call.

Some callers cannot call cudaMalloc -- a real-time sensor callback that must never
block, or a host whose device memory belongs to another allocator -- so this entry point
runs on a static device scratch array instead of a caller workspace.  The array is
shared by all calls and keeps the previous call's contents, so the check is made on two
calls in a row, the first on a larger cloud than the second.  Runs last (file name) and
on its own in a fresh process alike.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2102_11084_gb300 import synth, vg

pytestmark = pytest.mark.gpu

TOL_M = 1e-5  # centroid tolerance of the parity tests


def _compare(a, b):
    ka = a.keys.cpu().numpy().view(np.uint64)
    kb = b.keys.cpu().numpy().view(np.uint64)
    assert np.array_equal(ka, kb)
    assert torch.equal(a.counts, b.counts)
    assert torch.equal(a.origin, b.origin)
    err = (a.centroids.double() - b.centroids.double()).abs().max().item() if ka.size else 0.0
    assert err <= TOL_M
    if a.point_to_voxel is None or b.point_to_voxel is None:
        assert a.point_to_voxel is None and b.point_to_voxel is None
    else:
        assert torch.equal(a.point_to_voxel, b.point_to_voxel)


@pytest.mark.parametrize("method,p2v_first,p2v_second", [
    ("sort", True, True),            # wide layout twice (point_to_voxel)
    ("sort", False, False),          # the narrow layout (bucket grouping) twice
    ("sort", True, False),           # a wide large call, then a narrow small one
    ("sort_lsd", False, False),      # the narrow layout through the global radix sort
    ("sort_lsd", False, True),
])
def test_noalloc_matches_downsample_two_calls_in_a_row(method, p2v_first, p2v_second):
    frames = [(synth.rgbd_frame(1280, 720, seed=11, cx=639.5, cy=359.5), 0.02, p2v_first),
              (synth.rgbd_frame(640, 480, seed=12), 0.05, p2v_second)]
    for xyz_np, leaf, p2v in frames:
        xyz = torch.from_numpy(xyz_np).cuda()
        ref = vg.downsample(xyz, leaf, method=method, point_to_voxel=p2v)
        got = vg.downsample_noalloc(xyz, leaf, method=method, point_to_voxel=p2v)
        assert got.keys.numel() > 0
        _compare(got, ref)


def test_noalloc_rejects_hash_method():
    xyz = torch.from_numpy(synth.rgbd_frame(640, 480, seed=12)).cuda()
    with pytest.raises(RuntimeError, match="invalid argument"):
        vg.downsample_noalloc(xyz, 0.05, method="hash")


def test_noalloc_rejects_oversize_cloud():
    n = vg.NOALLOC_MAX_POINTS + 1
    xyz = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    out = torch.empty(16, dtype=torch.int64, device="cuda")
    st = vg.lib().vg_downsample_noalloc(
        ctypes.c_void_p(xyz.data_ptr()), n, ctypes.c_void_p(out.data_ptr()), ctypes.c_float(0.1),
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), 0, ctypes.c_void_p(out.data_ptr()), None, None, 0, None)
    assert st == vg.Status.INVALID_ARG
    assert vg.lib().vg_downsample_noalloc_scratch_bytes() >= vg.workspace_bytes(vg.NOALLOC_MAX_POINTS)
