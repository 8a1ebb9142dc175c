"""GPU parity of the persistent voxel map (vg_map_*): frames merged one insert at a time
into a device-resident table on a fixed lattice must extract exactly as one decimation
of all their points with the map's origin (Sec. II-C: every filtered camera cloud marks
the global map).  Keys and counts bit-exact; centroids within 1e-5 m; the extraction
is the same bits whatever the order and grouping of the inserts."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_11084_gb300 import synth, vg
from tests._parity import gpu_counts, gpu_keys, to_np

pytestmark = pytest.mark.gpu
ORIGIN = np.float32([-10.0, -10.0, -5.0])
LEAF = 0.05


def frames_and_poses(k=4, seed=40):
    frames = [synth.rgbd_frame(320, 240, seed=seed + f) for f in range(k)]
    poses, _ = synth.sensor_poses(k, seed=seed)
    bands = np.tile(np.float32([0.6, 1.0]), (k, 1))  # cuts these close-range scenes
    return frames, poses, bands


def same_bits(a, b):
    assert np.array_equal(gpu_keys(a.keys), gpu_keys(b.keys))
    assert np.array_equal(gpu_counts(a.counts), gpu_counts(b.counts))
    assert np.array_equal(to_np(a.centroids), to_np(b.centroids))


def test_inserts_equal_one_decimation_of_all_points():
    frames, poses, bands = frames_and_poses()
    m = vg.VoxelMap(200_000, ORIGIN, LEAF)
    for f, x in enumerate(frames):
        m.insert(torch.from_numpy(x).cuda(), poses=[poses[f].reshape(12)], z_limits=[bands[f]])
    got = m.extract()
    ref = oracle.map_contents(frames, LEAF, ORIGIN, poses, bands)
    assert ref.keys.size > 1000
    assert np.array_equal(gpu_keys(got.keys), ref.keys)
    assert np.array_equal(gpu_counts(got.counts), ref.counts)
    assert np.abs(to_np(got.centroids) - ref.centroids).max() <= 1e-5
    # the same bits whatever the grouping and order of the inserts
    m2 = vg.VoxelMap(200_000, ORIGIN, LEAF)
    m2.insert([torch.from_numpy(x).cuda() for x in frames[::-1]],
              poses=poses[::-1].reshape(-1, 12), z_limits=bands[::-1])
    same_bits(m2.extract(), got)
    # and the bits of the plain call on the posed, concatenated cloud with that origin
    cat = np.concatenate([oracle.pose(x, poses[f], bands[f]) for f, x in enumerate(frames)])
    solo = vg.downsample(torch.from_numpy(cat).cuda(), LEAF, torch.from_numpy(ORIGIN).cuda())
    same_bits(solo, got)
    m.close()
    m2.close()


def test_extract_leaves_the_map_and_inserts_continue():
    frames, _, _ = frames_and_poses(3, seed=50)
    m = vg.VoxelMap(200_000, ORIGIN, LEAF)
    m.insert(torch.from_numpy(frames[0]).cuda())
    first = m.extract()
    same_bits(m.extract(), first)
    m.insert([torch.from_numpy(x).cuda() for x in frames[1:]])
    ref = oracle.map_contents(frames, LEAF, ORIGIN)
    got = m.extract()
    assert np.array_equal(gpu_keys(got.keys), ref.keys)
    assert np.array_equal(gpu_counts(got.counts), ref.counts)
    assert np.abs(to_np(got.centroids) - ref.centroids).max() <= 1e-5
    m.clear()
    assert m.extract().keys.numel() == 0
    m.insert(torch.from_numpy(frames[2]).cuda())
    assert np.array_equal(gpu_keys(m.extract().keys),
                          oracle.map_contents(frames[2:], LEAF, ORIGIN).keys)
    m.close()


def test_points_outside_the_lattice_are_reported():
    m = vg.VoxelMap(10_000, ORIGIN, LEAF)
    x = np.float32([[0.0, 0.0, 0.0], [-20.0, 0.0, 0.0], [1.0, 1.0, 1.0]])
    m.insert(torch.from_numpy(x).cuda())
    with pytest.raises(vg.VGError) as e:
        m.extract()
    assert e.value.status == vg.Status.RANGE
    m.close()
