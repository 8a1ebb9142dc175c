"""Shared comparison helpers for the GPU parity tests (CUDA path vs CPU oracle).

Tolerances: keys, counts, order, V and point_to_voxel bit-exact; centroids within
1e-5 m (absolute) of the FP64 oracle.
"""
import numpy as np

CENTROID_TOL_M = 1e-5


def to_np(t):
    a = t.detach().cpu().numpy()
    return a


def gpu_keys(t):
    return to_np(t).view(np.uint64)


def gpu_counts(t):
    return to_np(t).view(np.uint32).astype(np.uint64)


def assert_decimation_equal(res, ref, *, check_p2v=True, tol=CENTROID_TOL_M):
    keys = gpu_keys(res.keys)
    assert keys.shape == ref.keys.shape, f"V {keys.shape[0]} != oracle {ref.keys.shape[0]}"
    assert np.array_equal(keys, ref.keys), "voxel keys/order differ"
    assert np.array_equal(gpu_counts(res.counts), ref.counts), "counts differ"
    c = to_np(res.centroids).astype(np.float64)
    if c.size:
        err = np.abs(c - ref.centroids).max()
        assert err <= tol, f"centroid max abs error {err:.3g} m > {tol}"
    assert np.array_equal(to_np(res.origin), ref.origin), "origin differs"
    if check_p2v and res.point_to_voxel is not None:
        assert np.array_equal(to_np(res.point_to_voxel), ref.point_to_voxel), "point_to_voxel differs"
