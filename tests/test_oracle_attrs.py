"""Pins of the oracle's readings R13 (mean 8-bit attributes per voxel, the RGB-D
camera's colour of Sec. II-B) and R14 (minimum points per voxel)."""
import numpy as np
import pytest

import oracle
from paper_2102_11084_gb300 import synth


def colours(n, channels, seed=0):
    return np.random.Generator(np.random.PCG64(seed)).integers(
        0, 256, size=(n, channels), dtype=np.uint8)


@pytest.mark.parametrize("channels", [1, 3, 4])
def test_means_against_brute_force(channels):
    x = synth.rgbd_frame(160, 120, seed=2)
    c = colours(x.shape[0], channels, seed=channels)
    r = oracle.downsample_attrs(x, 0.02, c)
    v = r.keys.shape[0]
    sums = np.zeros((v, channels))
    np.add.at(sums, r.point_to_voxel[r.point_to_voxel >= 0], c[r.point_to_voxel >= 0])
    want = (sums / r.counts[:, None].astype(np.float64)).astype(np.float32)
    assert np.array_equal(r.attrs, want)


def test_single_point_and_uniform_voxels_are_exact():
    leaf = 0.25
    pts = np.array([[0.1, 0.1, 0.1], [1.1, 0.1, 0.1], [1.2, 0.2, 0.2], [1.15, 0.05, 0.1]],
                   np.float32)
    col = np.array([[7, 200, 33], [10, 20, 30], [10, 20, 30], [10, 20, 30]], np.uint8)
    r = oracle.downsample_attrs(pts, leaf, col, origin_xyz=np.zeros(3, np.float32))
    assert r.keys.shape[0] == 2
    assert np.array_equal(r.attrs, np.float32([[7, 200, 33], [10, 20, 30]]))
    # 1/3 is not a binary32 value: the mean is the rounded FP64 quotient
    col2 = col.copy()
    col2[3] = [11, 20, 30]
    r2 = oracle.downsample_attrs(pts, leaf, col2, origin_xyz=np.zeros(3, np.float32))
    assert r2.attrs[1, 0] == np.float32(31.0 / 3.0)


@pytest.mark.parametrize("m", [1, 2, 3, 5, 10 ** 9])
def test_min_count_is_a_stable_filter(m):
    x = synth.random_cloud(4000, seed=12, extent=1.0, nan_frac=0.05)
    c = colours(x.shape[0], 3, seed=5)
    full = oracle.downsample_attrs(x, 0.08, c)
    r = oracle.downsample_attrs(x, 0.08, c, min_count=m)
    keep = full.counts >= m
    assert np.array_equal(r.keys, full.keys[keep])
    assert np.array_equal(r.counts, full.counts[keep])
    assert np.array_equal(r.centroids, full.centroids[keep])
    assert np.array_equal(r.attrs, full.attrs[keep])
    new_row = np.full(full.keys.shape[0], -1, np.int64)
    new_row[keep] = np.arange(int(keep.sum()))
    p = full.point_to_voxel
    want = np.where(p >= 0, new_row[np.maximum(p, 0)], -1)
    assert np.array_equal(r.point_to_voxel, want)
    assert int(r.counts.sum()) == int((r.point_to_voxel >= 0).sum())
    if m == 1:
        assert r.keys.shape[0] == full.keys.shape[0]
    if m == 10 ** 9:
        assert r.keys.shape[0] == 0
