"""The bucket grouping of the narrow sort path (method "sort" for 32-bit keys, and "auto"
from 2^22 points: partition passes over the top key bits, then every bucket reduced in
one block's shared memory through an occupancy bitmap of its low key bits): the same
rows as the
oracle and, bit for bit, as the global LSD radix sort with its segmented reduction
(method "sort_lsd"), for buckets of one key, of at most 8 and of more than 8 low bits,
one and two partition passes, buckets larger than a block stages (streamed in windows
of cells), buckets that are one voxel, a voxel of millions of points, skewed clouds,
batched frames and the pyramid."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_11084_gb300 import synth, vg
from tests._parity import assert_decimation_equal, gpu_counts, gpu_keys, to_np

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def same_rows(a, b):
    assert np.array_equal(gpu_keys(a.keys), gpu_keys(b.keys))
    assert np.array_equal(gpu_counts(a.counts), gpu_counts(b.counts))
    assert np.array_equal(to_np(a.centroids), to_np(b.centroids))


def check(x, leaf, origin=None):
    ref = oracle.downsample(x, leaf, origin)
    org = None if origin is None else torch.from_numpy(origin).cuda()
    got = vg.downsample(cuda(x), leaf, org, method="sort")
    assert_decimation_equal(got, ref, check_p2v=False)
    org2 = None if origin is None else torch.from_numpy(origin).cuda()
    same_rows(got, vg.downsample(cuda(x), leaf, org2, method="sort_lsd"))
    return got


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("n", [1, 2, 511, 512, 513, 3071, 3072, 3073, 4095, 4096, 4097,
                               8191, 8192, 8193, 100_000])
def test_sizes_around_tiles_and_stages(n):
    x = synth.random_cloud(n, seed=17 + n, extent=2.0, nan_frac=0.03)
    check(x, 0.02)


@pytest.mark.parametrize("edge,n", [(4, 50_000), (30, 50_000), (700, 120_000)])
def test_bucket_shifts(edge, n):
    # key widths of 6, 15 and 30 bits: one partition pass with buckets of one key, one
    # pass with a few low bits, and two passes with bitmaps of up to 2048 words
    x = (rng(edge).random((n, 3)) * edge * 0.02).astype(np.float32)
    check(x, 0.02, np.zeros(3, np.float32))


def test_bucket_larger_than_a_block():
    # a dense 0.4 m cluster puts ~150k points and ~8000 voxels in a few buckets (more
    # entries than a block stages, more cells than one window); a handful of far points
    # widen the key to 30 bits
    r = rng(5)
    cluster = (r.random((150_000, 3)) * 0.4).astype(np.float32)
    far = (r.random((50, 3)) * 20.0).astype(np.float32)
    x = np.concatenate([cluster, far])
    r.shuffle(x)
    check(x, 0.02)


def test_one_voxel_buckets_of_many_points():
    # 8 voxels of ~12k points each: every bucket is one voxel
    x = (rng(6).random((100_000, 3)) * 2.0).astype(np.float32)
    check(x, 1.0, np.zeros(3, np.float32))


def test_voxel_of_millions_of_points():
    # 2.2M points in one voxel: a streamed bucket whose one cell's sums exceed 32 bits
    x = (0.2 + rng(11).random((2_200_000, 3)) * 0.6).astype(np.float32)
    got = check(x, 1.0, np.zeros(3, np.float32))
    assert int(gpu_counts(got.counts)[0]) == 2_200_000


def test_all_points_in_one_voxel():
    x = np.full((40_000, 3), 0.5, np.float32) + \
        (rng(7).random((40_000, 3)) * 0.01).astype(np.float32)
    got = check(x, 0.1)
    assert int(gpu_counts(got.counts).sum()) == 40_000


def test_long_runs_inside_large_buckets():
    r = rng(8)
    centres = r.uniform(0, 0.3, size=(6, 3)).astype(np.float32)
    x = (centres[r.integers(0, 6, 120_000)] + r.normal(0, 0.002, size=(120_000, 3)))
    x = np.concatenate([x, r.random((20, 3)) * 10.0]).astype(np.float32)
    check(x, 0.01)


def test_fused_map_slice():
    x = synth.fused_map(400_000, 3)
    check(x, 0.02)


def test_batched_frames_match_full_sort():
    frames = [synth.rgbd_frame(320, 240, seed=500 + f) for f in range(9)]
    frames.append(np.zeros((0, 3), np.float32))
    frames.append(synth.random_cloud(5000, seed=9, extent=8.0))
    leaves = [0.02 + 0.01 * (f % 3) for f in range(len(frames))]
    a = vg.downsample_frames([cuda(f) for f in frames], leaves, method="sort")
    b = vg.downsample_frames([cuda(f) for f in frames], leaves, method="sort_lsd")
    assert list(a.offsets) == list(b.offsets)
    same_rows(a, b)
    for f, x in enumerate(frames):
        ref = oracle.downsample(x, leaves[f])
        lo, hi = int(a.offsets[f]), int(a.offsets[f + 1])
        assert np.array_equal(gpu_keys(a.keys[lo:hi]), ref.keys)
        assert np.array_equal(gpu_counts(a.counts[lo:hi]), ref.counts)


def test_pyramid_on_the_bucket_grouping():
    x = synth.random_cloud(80_000, seed=21, extent=3.0)
    p = vg.pyramid(cuda(x), 0.02, 3, method="sort")
    q = vg.pyramid(cuda(x), 0.02, 3, method="sort_lsd")
    for lvl in range(3):
        same_rows(p[lvl], q[lvl])
    ref, _ = oracle.pyramid(x, 0.02, 3)
    for lvl in range(3):
        assert np.array_equal(gpu_keys(p[lvl].keys), ref[lvl][0])
        assert np.array_equal(gpu_counts(p[lvl].counts), ref[lvl][2])


def test_frames_straddling_partition_tiles():
    # frames of 1 to 5000 points: the key kernel's chunks and the partition passes' tiles
    # of 4096 entries hold many frames
    r = rng(31)
    sizes = [1, 2, 3, 4095, 4097, 1, 0, 5000, 7, 4096, 13, 2049, 1, 1, 1]
    frames = [(r.random((m, 3)) * 3.0).astype(np.float32) for m in sizes]
    leaves = [0.05 + 0.01 * (f % 4) for f in range(len(frames))]
    a = vg.downsample_frames([cuda(f) for f in frames], leaves, method="sort")
    b = vg.downsample_frames([cuda(f) for f in frames], leaves, method="sort_lsd")
    assert list(a.offsets) == list(b.offsets)
    same_rows(a, b)
    for f, x in enumerate(frames):
        ref = oracle.downsample(x, leaves[f])
        lo, hi = int(a.offsets[f]), int(a.offsets[f + 1])
        assert np.array_equal(gpu_keys(a.keys[lo:hi]), ref.keys)
        assert np.array_equal(gpu_counts(a.counts[lo:hi]), ref.counts)


@pytest.mark.parametrize("n", [307_200, 4_500_000])
def test_auto_picks_by_size_and_matches_both_groupings(n):
    # "auto" takes the global radix sort below 2^22 points and the bucket grouping from
    # there: its rows are bit-identical to both
    x = synth.fused_map(n, seed=41)
    auto = vg.downsample(cuda(x), 0.02)
    same_rows(auto, vg.downsample(cuda(x), 0.02, method="sort"))
    same_rows(auto, vg.downsample(cuda(x), 0.02, method="sort_lsd"))
