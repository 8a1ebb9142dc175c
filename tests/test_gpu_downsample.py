"""GPU parity of vg_downsample (through the C ABI) against the CPU oracle.

Keys, counts, order, V and point_to_voxel must be bit-exact; centroids within 1e-5 m.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_11084_gb300 import synth, vg
from tests._parity import assert_decimation_equal, gpu_counts, gpu_keys, to_np

pytestmark = pytest.mark.gpu


def run(xyz_np, leaf, origin=None, **kw):
    xyz = torch.from_numpy(np.ascontiguousarray(xyz_np, np.float32)).cuda()
    o = None if origin is None else torch.from_numpy(np.asarray(origin, np.float32)).cuda()
    return vg.downsample(xyz, leaf, o, **kw)


@pytest.mark.parametrize("leaf", [0.05])
def test_rgbd_640x480(leaf):
    xyz = synth.rgbd_frame(640, 480, seed=0)
    ref = oracle.downsample(xyz, leaf)
    res = run(xyz, leaf, point_to_voxel=True)
    assert_decimation_equal(res, ref)


@pytest.mark.parametrize("leaf", [0.01, 0.02, 0.05, 0.1])
def test_rgbd_1280x720_sweep(leaf):
    xyz = synth.rgbd_frame(1280, 720, seed=0, cx=639.5, cy=359.5)
    ref = oracle.downsample(xyz, leaf)
    res = run(xyz, leaf, point_to_voxel=True)
    assert_decimation_equal(res, ref)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 127, 1000, 2047, 2048, 2049, 4095, 4096, 4097,
                               8191, 12289, 65537])
def test_ragged_sizes(n):
    xyz = synth.random_cloud(n, seed=n, extent=3.0, nan_frac=0.1, inf_frac=0.02)
    ref = oracle.downsample(xyz, 0.07)
    res = run(xyz, 0.07, point_to_voxel=True)
    assert_decimation_equal(res, ref)


def test_empty_and_all_invalid():
    res = run(np.zeros((0, 3), np.float32), 0.1)
    assert res.keys.numel() == 0
    bad = np.full((1000, 3), np.nan, np.float32)
    bad[::3, 1] = 1.0
    res = run(bad, 0.1, point_to_voxel=True)
    assert res.keys.numel() == 0
    assert (to_np(res.point_to_voxel) == -1).all()
    assert (to_np(res.origin) == 0).all()


def test_single_voxel_long_run():
    # every point in one voxel: the run spans many tiles of the segmented reduction
    rng = np.random.Generator(np.random.PCG64(3))
    xyz = (rng.uniform(0.0, 0.99, size=(300_000, 3)) + 5.0).astype(np.float32)
    ref = oracle.downsample(xyz, 4.0, np.zeros(3, np.float32))
    res = run(xyz, 4.0, origin=np.zeros(3))
    assert_decimation_equal(res, ref)
    assert int(gpu_counts(res.counts)[0]) == 300_000


def test_few_voxels_many_points():
    xyz = synth.random_cloud(200_000, 8, extent=1.0, nan_frac=0.05, clusters=5,
                             cluster_sigma=0.05)
    ref = oracle.downsample(xyz, 0.3)
    res = run(xyz, 0.3, point_to_voxel=True)
    assert_decimation_equal(res, ref)


def test_given_origin_and_faces():
    leaf = 0.25
    o = np.array([1.0, -2.0, 0.5], np.float32)
    k = np.random.Generator(np.random.PCG64(4)).integers(0, 50, size=(20_000, 3))
    pts = (o + k.astype(np.float32) * np.float32(leaf)).astype(np.float32)  # exactly on faces
    ref = oracle.downsample(pts, leaf, o)
    res = run(pts, leaf, origin=o, point_to_voxel=True)
    assert_decimation_equal(res, ref)


def test_near_face_keys_non_power_of_two_leaf():
    rng = np.random.Generator(np.random.PCG64(21))
    leaf = 0.013
    o = rng.uniform(-3, 3, size=3).astype(np.float32)
    k = rng.integers(0, 400, size=(50_000, 3))
    pts = (o.astype(np.float64) + k * leaf).astype(np.float32)
    for s in range(3):
        m = rng.integers(-1, 2, size=pts.shape)
        pts = np.where(m > 0, np.nextafter(pts, np.float32(np.inf)),
                       np.where(m < 0, np.nextafter(pts, np.float32(-np.inf)), pts)).astype(np.float32)
    pts = pts[(pts >= o).all(axis=1)]
    ref = oracle.downsample(pts, leaf, o)
    res = run(pts, leaf, origin=o)
    assert_decimation_equal(res, ref)


def test_misaligned_input():
    xyz = synth.random_cloud(10_001, 12, extent=2.0)
    big = torch.from_numpy(np.concatenate([np.zeros((1, 3), np.float32), xyz])).cuda()
    view = big.view(-1)[3:].view(-1, 3)  # 12-byte offset: not 16-byte aligned
    assert view.data_ptr() % 16 != 0
    res = vg.downsample(view, 0.05)
    assert_decimation_equal(res, oracle.downsample(xyz, 0.05), check_p2v=False)


def test_deterministic_bits():
    xyz = synth.rgbd_frame(320, 240, seed=9)
    a = run(xyz, 0.02)
    b = run(xyz, 0.02)
    assert torch.equal(a.keys, b.keys) and torch.equal(a.counts, b.counts)
    assert torch.equal(a.centroids.view(torch.int32), b.centroids.view(torch.int32))


def test_range_error_is_reported():
    xyz = np.array([[0.0, 0.0, 0.0], [1e6, 0.0, 0.0]], np.float32)
    with pytest.raises(vg.VGError) as e:
        run(xyz, 0.01)
    assert e.value.status == vg.Status.RANGE


def test_capacity_error_is_reported():
    xyz = torch.from_numpy(synth.random_cloud(5000, 2, extent=1.0, nan_frac=0.0)).cuda()
    buf = vg.alloc_buffers(5000, "cuda", cap=10)
    vg.downsample_into(xyz, 0.05, buf, origin_from_min=True, cap=10)
    torch.cuda.synchronize()
    assert int(buf.error.item()) == vg.Status.CAPACITY
    ref = oracle.downsample(synth.random_cloud(5000, 2, extent=1.0, nan_frac=0.0), 0.05)
    assert np.array_equal(gpu_keys(buf.keys[:10]), ref.keys[:10])


@pytest.fixture(scope="module")
def fused_map_50m():
    return synth.fused_map(50_000_000, seed=0)


@pytest.mark.parametrize("leaf", [0.02, 0.1])
def test_fused_map_full_size(fused_map_50m, leaf):
    """The 50M-point map cloud at both of its leaves, through the library's default
    (the bucket grouping at this size): origin, every key, count and the order exactly,
    against the oracle's per-point keys; every centroid within 1e-5 m of the FP64 mean of
    its member points; at 0.02 m also the global radix sort's rows, bit for bit."""
    xyz = fused_map_50m
    res = run(xyz, leaf)
    k_gpu = gpu_keys(res.keys)
    c_gpu = gpu_counts(res.counts)
    o = to_np(res.origin)
    o_ref, nvalid = oracle.origin(xyz)
    assert np.array_equal(o, o_ref)
    keys, _, valid, st = oracle.keys(xyz, o_ref, leaf)
    assert st == 0
    kv = keys[valid]
    uniq, inv, cnt = np.unique(kv, return_inverse=True, return_counts=True)
    del kv
    assert np.array_equal(k_gpu, uniq)
    assert np.array_equal(c_gpu, cnt.astype(np.uint64))
    cent = to_np(res.centroids).astype(np.float64)
    pts = xyz[valid]
    err = 0.0
    for a in range(3):
        mean = np.bincount(inv, weights=pts[:, a].astype(np.float64),
                           minlength=uniq.shape[0]) / cnt
        err = max(err, float(np.abs(cent[:, a] - mean).max()))
    assert err <= 1e-5, err
    if leaf == 0.02:
        other = run(xyz, leaf, method="sort_lsd")
        assert torch.equal(other.keys, res.keys) and torch.equal(other.counts, res.counts)
        assert torch.equal(other.centroids.view(torch.int32), res.centroids.view(torch.int32))


@pytest.mark.parametrize("top,hi", [((2047, 2047, 1023), (2048, 2048, 1024)),
                                    ((2046, 2047, 1023), (2047, 2048, 1024))])
def test_all_ones_32bit_key(top, hi):
    """A voxel whose 32-bit Morton key is all ones (first case) sits next to invalid rows,
    whose sort key is all ones too; one just below it (second case) lets the extents pick
    the 32-bit sort layout.  Both must drop exactly the invalid rows."""
    leaf = 2.0 ** -6
    rng = np.random.Generator(np.random.PCG64(11))
    idx = rng.integers(0, hi, size=(6000, 3))
    idx[:40] = top
    xyz = ((idx + rng.uniform(0.1, 0.9, size=idx.shape)) * leaf).astype(np.float32)
    xyz[40 + rng.choice(5960, 400, replace=False)] = np.nan
    ref = oracle.downsample(xyz, leaf, np.zeros(3, np.float32))
    res = run(xyz, leaf, origin=(0.0, 0.0, 0.0))
    assert_decimation_equal(res, ref)
    ix, iy, iz = top
    want = sum(((ix >> b) & 1) << (3 * b) | ((iy >> b) & 1) << (3 * b + 1) |
               ((iz >> b) & 1) << (3 * b + 2) for b in range(11))
    assert int(ref.keys[-1]) == want and int(ref.counts[-1]) == 40
