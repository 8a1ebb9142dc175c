"""GPU parity of the hash grouping path (VG_METHOD_HASH) against the oracle, and its
bit-equality with the sort path (same key, same fixed-point accumulator)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_11084_gb300 import synth, vg
from tests._parity import assert_decimation_equal

pytestmark = pytest.mark.gpu


def run(xyz_np, leaf, method, origin=None, p2v=True):
    xyz = torch.from_numpy(np.ascontiguousarray(xyz_np, np.float32)).cuda()
    o = None if origin is None else torch.from_numpy(np.asarray(origin, np.float32)).cuda()
    return vg.downsample(xyz, leaf, o, method=method, point_to_voxel=p2v)


@pytest.mark.parametrize("leaf", [0.02, 0.05, 0.1])
def test_hash_rgbd_640x480(leaf):
    xyz = synth.rgbd_frame(640, 480, seed=0)
    assert_decimation_equal(run(xyz, leaf, "hash"), oracle.downsample(xyz, leaf))


@pytest.mark.parametrize("n", [1, 5, 1000, 4097, 65537])
def test_hash_ragged(n):
    xyz = synth.random_cloud(n, seed=100 + n, extent=3.0, nan_frac=0.1, inf_frac=0.02)
    assert_decimation_equal(run(xyz, 0.07, "hash"), oracle.downsample(xyz, 0.07))


def test_hash_dense_voxels():
    # many points per voxel: heavy slot contention, long warp groups
    xyz = synth.random_cloud(400_000, 3, extent=1.0, nan_frac=0.05, clusters=3, cluster_sigma=0.02)
    assert_decimation_equal(run(xyz, 0.5, "hash"), oracle.downsample(xyz, 0.5))


def test_hash_empty_and_invalid():
    assert run(np.zeros((0, 3), np.float32), 0.1, "hash", p2v=False).keys.numel() == 0
    bad = np.full((777, 3), np.nan, np.float32)
    r = run(bad, 0.1, "hash")
    assert r.keys.numel() == 0 and (r.point_to_voxel.cpu().numpy() == -1).all()


@pytest.mark.parametrize("leaf", [0.01, 0.1])
def test_sort_and_hash_bit_identical(leaf):
    xyz = synth.rgbd_frame(1280, 720, seed=2, cx=639.5, cy=359.5)
    a = run(xyz, leaf, "sort")
    b = run(xyz, leaf, "hash")
    assert torch.equal(a.keys, b.keys) and torch.equal(a.counts, b.counts)
    assert torch.equal(a.centroids.view(torch.int32), b.centroids.view(torch.int32))
    assert torch.equal(a.point_to_voxel, b.point_to_voxel)
