"""GPU parity of posed frames (vg_downsample_frames_posed): sensor pose p' = R p + t and
the height band [z_min, z_max] fused into the first read of every point, against the
oracle's reading R12 (Sec. II-C: clouds are taken into the global frame, where the
filter limits the height).  Keys, counts, order, V and point_to_voxel bit-exact;
centroids within 1e-5 m."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_11084_gb300 import synth, vg
from tests._parity import assert_decimation_equal, gpu_counts, gpu_keys, to_np

pytestmark = pytest.mark.gpu


def random_pose(seed, shift=2.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.normal(size=4)
    w, a, b, c = q / np.linalg.norm(q)
    R = np.array([[1 - 2 * (b * b + c * c), 2 * (a * b - c * w), 2 * (a * c + b * w)],
                  [2 * (a * b + c * w), 1 - 2 * (a * a + c * c), 2 * (b * c - a * w)],
                  [2 * (a * c - b * w), 2 * (b * c + a * w), 1 - 2 * (a * a + b * b)]])
    t = rng.uniform(-shift, shift, size=(3, 1))
    return np.concatenate([R, t], axis=1).astype(np.float32)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("method", ["sort", "hash"])
@pytest.mark.parametrize("p2v", [False, True])
def test_posed_rgbd_frame(method, p2v):
    xyz = synth.rgbd_frame(640, 480, seed=3)
    rt = random_pose(21)
    band = np.float32([-1.5, 2.0])
    ref = oracle.downsample_posed(xyz, 0.05, rt, band)
    assert 0 < ref.counts.sum() < np.isfinite(xyz).all(axis=1).sum()  # the band cuts
    res = vg.downsample(cuda(xyz), 0.05, pose=rt, z_limits=band, method=method,
                        point_to_voxel=p2v)
    assert_decimation_equal(res, ref)


def test_identity_pose_is_the_plain_call():
    xyz = synth.rgbd_frame(320, 240, seed=4)
    eye = np.eye(3, 4, dtype=np.float32)
    a = vg.downsample(cuda(xyz), 0.03, pose=eye)
    b = vg.downsample(cuda(xyz), 0.03)
    assert np.array_equal(gpu_keys(a.keys), gpu_keys(b.keys))
    assert np.array_equal(gpu_counts(a.counts), gpu_counts(b.counts))
    assert np.array_equal(to_np(a.centroids), to_np(b.centroids))


def test_band_only_and_empty_band():
    xyz = synth.rgbd_frame(320, 240, seed=5)
    band = np.float32([1.0, 3.0])
    ref = oracle.downsample_posed(xyz, 0.04, None, band)
    assert_decimation_equal(vg.downsample(cuda(xyz), 0.04, z_limits=band), ref)
    res = vg.downsample(cuda(xyz), 0.04, z_limits=np.float32([100.0, 101.0]),
                        point_to_voxel=True)
    assert res.keys.numel() == 0 and (to_np(res.point_to_voxel) == -1).all()


@pytest.mark.parametrize("method", ["sort", "hash"])
def test_posed_batch_matches_per_frame_oracle(method):
    rng = np.random.Generator(np.random.PCG64(8))
    frames = [synth.rgbd_frame(320, 240, seed=60 + f) for f in range(6)]
    frames = [x[: int(rng.integers(5_000, x.shape[0]))] for x in frames]
    frames[2] = frames[2][:0]  # an empty frame in the middle
    leaves = np.float32([0.02, 0.05, 0.1, 0.03, 0.05, 0.02])
    poses = np.stack([random_pose(100 + f, shift=5.0) for f in range(6)])
    # each frame's band keeps a different slice of its posed heights
    bands = np.zeros((6, 2), np.float32)
    for f, (lo, hi) in enumerate([(10, 90), (0, 50), (30, 100), (5, 60), (40, 95), (0, 100)]):
        z = oracle.pose(frames[f], poses[f])[:, 2]
        z = z[np.isfinite(z)]
        bands[f] = np.percentile(z, [lo, hi]) if z.size else (0.0, 1.0)
    out = vg.downsample_frames([cuda(x) for x in frames], leaves, method=method, poses=poses,
                               z_limits=bands, point_to_voxel=True)
    p2v = to_np(out.point_to_voxel)
    start = 0
    for f, x in enumerate(frames):
        ref = oracle.downsample_posed(x, float(leaves[f]), poses[f], bands[f])
        got = out.frame(f)
        assert np.array_equal(gpu_keys(got.keys), ref.keys), f
        assert np.array_equal(gpu_counts(got.counts), ref.counts), f
        if ref.keys.size:
            assert np.abs(to_np(got.centroids) - ref.centroids).max() <= 1e-5, f
        assert np.array_equal(to_np(got.origin), ref.origin), f
        local = p2v[start:start + x.shape[0]]
        want = np.where(ref.point_to_voxel < 0, -1, ref.point_to_voxel + out.offsets[f])
        assert np.array_equal(local, want), f
        start += x.shape[0]
    # a frame decimated alone gives the same bits as inside the batch
    solo = vg.downsample(cuda(frames[4]), float(leaves[4]), pose=poses[4], z_limits=bands[4],
                         method=method)
    assert np.array_equal(gpu_keys(solo.keys), gpu_keys(out.frame(4).keys))
    assert np.array_equal(to_np(solo.centroids), to_np(out.frame(4).centroids))
