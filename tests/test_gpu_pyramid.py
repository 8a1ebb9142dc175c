"""GPU pyramid (vg_pyramid) against the oracle's count-weighted key>>3 merge, and the
bit-exact pyramid invariant: level k keys/counts == direct decimation at 2^k * leaf."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_11084_gb300 import synth, vg
from tests._parity import CENTROID_TOL_M, gpu_counts, gpu_keys, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("w,h,leaf,levels", [(1280, 720, 0.01, 4), (320, 240, 0.02, 3),
                                             (640, 480, 0.05, 1)])
def test_pyramid_levels(w, h, leaf, levels):
    xyz = synth.rgbd_frame(w, h, seed=0, cx=(w - 1) / 2, cy=(h - 1) / 2)
    pyr = vg.pyramid(torch.from_numpy(xyz).cuda(), leaf, levels, point_to_voxel=True)
    ref_levels, d0 = oracle.pyramid(xyz, leaf, levels)
    assert np.array_equal(to_np(pyr[0].point_to_voxel), d0.point_to_voxel)
    for k in range(levels):
        keys, cents, counts = ref_levels[k]
        assert np.array_equal(gpu_keys(pyr[k].keys), keys), f"level {k} keys"
        assert np.array_equal(gpu_counts(pyr[k].counts), counts), f"level {k} counts"
        err = np.abs(to_np(pyr[k].centroids).astype(np.float64) - cents).max()
        assert err <= CENTROID_TOL_M, (k, err)
        direct = oracle.downsample(xyz, float(np.float32(2 ** k) * np.float32(leaf)), d0.origin)
        assert np.array_equal(gpu_keys(pyr[k].keys), direct.keys)
        assert np.array_equal(gpu_counts(pyr[k].counts), direct.counts)


def test_pyramid_level_equals_gpu_direct():
    xyz = torch.from_numpy(synth.rgbd_frame(640, 480, seed=7)).cuda()
    pyr = vg.pyramid(xyz, 0.01, 4)
    for k in range(4):
        d = vg.downsample(xyz, float(np.float32(2 ** k) * np.float32(0.01)), pyr[0].origin)
        assert torch.equal(pyr[k].keys, d.keys) and torch.equal(pyr[k].counts, d.counts)
        assert (pyr[k].centroids - d.centroids).abs().max().item() <= CENTROID_TOL_M


def test_pyramid_empty():
    pyr = vg.pyramid(torch.zeros((0, 3), device="cuda"), 0.1, 3)
    assert all(l.keys.numel() == 0 for l in pyr)
