"""GPU backward (vg_downsample_backward, VoxelDownsample) against the oracle's analytic
gradient and central finite differences of the FP64 oracle loss."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_11084_gb300 import synth, vg
from tests._parity import to_np

pytestmark = pytest.mark.gpu


def test_backward_kernel_matches_oracle():
    xyz = synth.rgbd_frame(640, 480, seed=0)
    leaf = 0.05
    ref = oracle.downsample(xyz, leaf)
    rng = np.random.Generator(np.random.PCG64(1))
    grad_c = rng.normal(size=ref.centroids.shape)
    want = oracle.backward(grad_c, ref.counts, ref.point_to_voxel)
    r = vg.downsample(torch.from_numpy(xyz).cuda(), leaf, point_to_voxel=True)
    g = vg.backward(torch.from_numpy(grad_c.astype(np.float32)).cuda(), r.counts, r.point_to_voxel)
    got = to_np(g).astype(np.float64)
    want32 = oracle.backward(grad_c.astype(np.float32).astype(np.float64), ref.counts,
                             ref.point_to_voxel)
    assert np.allclose(got, want32, rtol=1e-6, atol=0)
    assert (got[ref.point_to_voxel < 0] == 0).all()
    assert np.allclose(got, want, rtol=1e-6, atol=1e-6)


def test_autograd_loss_gradient_vs_finite_differences():
    """Mean squared centroid loss on the 640x480 frame at leaf 0.05 m (307,200 points)."""
    xyz_np = synth.rgbd_frame(640, 480, seed=0)
    leaf = 0.05
    ref = oracle.downsample(xyz_np, leaf)
    V = len(ref.keys)
    rng = np.random.Generator(np.random.PCG64(2))
    targets = ref.centroids + rng.normal(size=ref.centroids.shape) * 0.01
    xyz = torch.from_numpy(xyz_np).cuda().requires_grad_(True)
    cents, keys, counts = vg.VoxelDownsample.apply(xyz, leaf, None)
    t = torch.from_numpy(targets.astype(np.float32)).cuda()
    loss = ((cents - t) ** 2).mean()
    loss.backward()
    g = to_np(xyz.grad).astype(np.float64)
    analytic = oracle.backward(oracle.loss_grad_centroids(ref.centroids, targets), ref.counts,
                               ref.point_to_voxel)
    valid = ref.point_to_voxel >= 0
    # Each entry is 2 (c - t) / (3 V n): a GPU centroid within the 1e-5 m parity tolerance
    # of the FP64 one, plus the binary32 rounding of the targets (< 1e-6 m here), bounds
    # the difference by 2 * 1.1e-5 / (3 V n) -- an absolute bound per point.
    n_of = np.zeros(len(xyz_np))
    n_of[valid] = ref.counts[ref.point_to_voxel[valid]].astype(np.float64)
    bound = 2 * 1.1e-5 / (3 * V * np.maximum(n_of, 1))
    assert (np.abs(g - analytic)[valid] <= bound[valid, None]).all()
    assert (g[~valid] == 0).all()
    # central differences of the FP64 oracle loss on points >= 1e-3 leaf from faces
    x64 = xyz_np.astype(np.float64)
    ijk = np.floor((x64[valid] - ref.origin.astype(np.float64)) / leaf)
    frac = np.zeros_like(x64)
    frac[valid] = (x64[valid] - ref.origin.astype(np.float64)) / leaf - ijk
    far = np.nonzero(valid & ((frac > 1e-3) & (frac < 1 - 1e-3)).all(axis=1))[0]
    h = 1e-4 * leaf
    for i in rng.choice(far, size=25, replace=False):
        for a in range(3):
            xp, xm = x64.copy(), x64.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = (oracle.centroid_loss(xp, ref.point_to_voxel, V, targets) -
                  oracle.centroid_loss(xm, ref.point_to_voxel, V, targets)) / (2 * h)
            assert abs(fd - g[i, a]) <= bound[i] + 1e-6 * abs(fd), (i, a, fd, g[i, a])
