"""The narrow layout (32-bit keys, packed offsets, chosen when no point_to_voxel is
asked for): the same rows as the oracle and, bit for bit, as the wide layout (forced
here by asking for point_to_voxel), across tile edges, long runs of one key,
single-digit keys and batched frames."""
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


@pytest.mark.parametrize("n", [2, 255, 1023, 1024, 1025, 3000, 4097, 65537, 300_001])
@pytest.mark.parametrize("extent", [0.6, 5.0])
def test_narrow_matches_oracle_and_wide(n, extent):
    x = synth.random_cloud(n, seed=n + int(extent), extent=extent, nan_frac=0.05)
    ref = oracle.downsample(x, 0.02)
    narrow = vg.downsample(cuda(x), 0.02)
    assert_decimation_equal(narrow, ref, check_p2v=False)
    same_rows(narrow, vg.downsample(cuda(x), 0.02, point_to_voxel=True))


def test_runs_longer_than_many_tiles():
    # a few dense voxels: runs of tens of thousands of entries cross many tiles
    rng = np.random.Generator(np.random.PCG64(2))
    centres = rng.uniform(0, 3, size=(12, 3)).astype(np.float32)
    x = (centres[rng.integers(0, 12, 200_000)] +
         rng.normal(0, 0.01, size=(200_000, 3))).astype(np.float32)
    ref = oracle.downsample(x, 0.05)
    narrow = vg.downsample(cuda(x), 0.05)
    assert_decimation_equal(narrow, ref, check_p2v=False)
    same_rows(narrow, vg.downsample(cuda(x), 0.05, point_to_voxel=True))


def test_one_and_two_digit_keys():
    # every key below 256 (one radix pass), and keys just above it
    rng = np.random.Generator(np.random.PCG64(3))
    for edge in (4, 6):
        x = (rng.random((20_000, 3)) * edge).astype(np.float32)
        ref = oracle.downsample(x, 1.0, np.zeros(3, np.float32))
        res = vg.downsample(cuda(x), 1.0, torch.zeros(3, device="cuda"))
        assert_decimation_equal(res, ref, check_p2v=False)


def test_batched_frames_narrow():
    rng = np.random.Generator(np.random.PCG64(4))
    frames = [synth.rgbd_frame(320, 240, seed=300 + f) for f in range(7)]
    frames = [x[: int(rng.integers(0, x.shape[0]))] for x in frames]
    leaves = np.float32([0.01, 0.02, 0.05, 0.1, 0.02, 0.03, 0.01])
    out = vg.downsample_frames([cuda(x) for x in frames], leaves)
    for f, x in enumerate(frames):
        ref = oracle.downsample(x, float(leaves[f]))
        got = out.frame(f)
        assert np.array_equal(gpu_keys(got.keys), ref.keys), f
        assert np.array_equal(gpu_counts(got.counts), ref.counts), f
        if ref.keys.size:
            assert np.abs(to_np(got.centroids) - ref.centroids).max() <= 1e-5, f
