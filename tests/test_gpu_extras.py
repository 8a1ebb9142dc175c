"""GPU parity of the voxel extras (vg_downsample_frames_ex): per-voxel means of 8-bit
attributes (reading R13; the camera is RGB-D, Sec. II-B) and the minimum points per
voxel (reading R14).  Attribute means are bit-exact (exact integer sums, one FP64
division, rounded to float32 on both sides); keys, counts, offsets and point_to_voxel
bit-exact; centroids within 1e-5 m."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_11084_gb300 import synth, vg
from tests._parity import gpu_counts, gpu_keys, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-5


def cuda(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype)).cuda()


def colours(n, channels, seed):
    return np.random.Generator(np.random.PCG64(seed)).integers(
        0, 256, size=(n, channels), dtype=np.uint8)


def check(res, ref, p2v=True):
    assert np.array_equal(gpu_keys(res.keys), ref.keys)
    assert np.array_equal(gpu_counts(res.counts), ref.counts)
    if ref.keys.size:
        assert np.abs(to_np(res.centroids) - ref.centroids).max() <= TOL
    if ref.attrs.shape[1]:
        assert np.array_equal(to_np(res.attrs), ref.attrs)
    if p2v:
        assert np.array_equal(to_np(res.point_to_voxel), ref.point_to_voxel)


@pytest.mark.parametrize("channels", [1, 3, 4])
def test_attribute_means_rgbd(channels):
    xyz = synth.rgbd_frame(640, 480, seed=7)
    col = colours(xyz.shape[0], channels, seed=channels)
    ref = oracle.downsample_attrs(xyz, 0.05, col)
    res = vg.downsample(cuda(xyz), 0.05, attrs=cuda(col, np.uint8), point_to_voxel=True)
    check(res, ref)


def test_attribute_mean_of_a_voxel_spanning_many_tiles():
    rng = np.random.Generator(np.random.PCG64(4))
    xyz = (0.5 + 0.4 * rng.random((20000, 3))).astype(np.float32)
    xyz[rng.choice(20000, 500, replace=False)] = np.nan
    col = colours(20000, 3, seed=9)
    ref = oracle.downsample_attrs(xyz, 1.0, col, origin_xyz=np.zeros(3, np.float32))
    res = vg.downsample(cuda(xyz), 1.0, torch.zeros(3, device="cuda"),
                        attrs=cuda(col, np.uint8), point_to_voxel=True)
    assert ref.keys.shape[0] == 1
    check(res, ref)


@pytest.mark.parametrize("method", ["sort", "hash"])
@pytest.mark.parametrize("m", [2, 3, 6, 10 ** 6])
def test_min_count(method, m):
    xyz = synth.rgbd_frame(640, 480, seed=8)
    ref = oracle.downsample_attrs(xyz, 0.02, None, min_count=m)
    res = vg.downsample(cuda(xyz), 0.02, min_count=m, method=method, point_to_voxel=True)
    check(res, ref)


def test_min_count_with_attrs_on_ragged_sizes():
    for n in (1, 1023, 1024, 1025, 5000):
        xyz = synth.random_cloud(n, seed=n, extent=0.6, nan_frac=0.1)
        col = colours(n, 2, seed=n)
        ref = oracle.downsample_attrs(xyz, 0.1, col, min_count=2)
        res = vg.downsample(cuda(xyz), 0.1, attrs=cuda(col, np.uint8), min_count=2,
                            point_to_voxel=True)
        check(res, ref)


def test_posed_batch_with_attrs_and_min_count():
    rng = np.random.Generator(np.random.PCG64(12))
    frames = [synth.rgbd_frame(320, 240, seed=80 + f) for f in range(5)]
    frames = [x[: int(rng.integers(3_000, x.shape[0]))] for x in frames]
    cols = [colours(x.shape[0], 3, seed=200 + f) for f, x in enumerate(frames)]
    leaves = np.float32([0.02, 0.05, 0.03, 0.1, 0.04])
    poses, bands = synth.sensor_poses(5, seed=3)
    out = vg.downsample_frames([cuda(x) for x in frames], leaves,
                               poses=poses.reshape(5, 12), z_limits=bands,
                               attrs=[cuda(c, np.uint8) for c in cols], min_count=2,
                               point_to_voxel=True)
    p2v = to_np(out.point_to_voxel)
    start = 0
    for f, x in enumerate(frames):
        ref = oracle.downsample_attrs(x, float(leaves[f]), cols[f], min_count=2,
                                      pose_rt=poses[f], z_limits=bands[f])
        got = out.frame(f)
        assert np.array_equal(gpu_keys(got.keys), ref.keys), f
        assert np.array_equal(gpu_counts(got.counts), ref.counts), f
        assert np.array_equal(to_np(got.attrs), ref.attrs), f
        if ref.keys.size:
            assert np.abs(to_np(got.centroids) - ref.centroids).max() <= TOL, f
        local = p2v[start:start + x.shape[0]]
        want = np.where(ref.point_to_voxel < 0, -1, ref.point_to_voxel + out.offsets[f])
        assert np.array_equal(local, want), f
        start += x.shape[0]


def test_attrs_need_the_sort_path():
    xyz = synth.rgbd_frame(160, 120, seed=1)
    col = colours(xyz.shape[0], 3, seed=1)
    with pytest.raises(vg.VGError) as e:
        vg.downsample(cuda(xyz), 0.05, attrs=cuda(col, np.uint8), method="hash")
    assert e.value.status == vg.Status.INVALID_ARG
