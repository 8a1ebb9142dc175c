"""The single-frame bin grouping (method "frame", VG_SORT_FRAME): keys counted into bins
of 2^12 consecutive keys, scattered once, every bin reduced densely in shared memory, row
offsets by a chained scan over units of bins.  Its rows must be the oracle's (keys,
counts and order bit-exact, centroids within 1e-5 m) and, bit for bit, those of the
global radix sort ("sort_lsd"), across key widths from one bin (keys under 2^12) to units
of many bins (keys of up to 32 bits), ragged sizes, cells of more than 2048 points, posed
frames and the one-frame plan with its CUDA graph."""
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
    assert np.array_equal(to_np(a.centroids).view(np.int32), to_np(b.centroids).view(np.int32))


def check(x, leaf, origin=None):
    org = None if origin is None else cuda(origin)
    got = vg.downsample(cuda(x), leaf, org, method="frame")
    assert_decimation_equal(got, oracle.downsample(x, leaf, origin), check_p2v=False)
    same_rows(got, vg.downsample(cuda(x), leaf, None if origin is None else cuda(origin),
                                 method="sort_lsd"))
    return got


def test_rgbd_640x480():
    check(synth.rgbd_frame(640, 480, seed=0), 0.05)


@pytest.mark.parametrize("leaf", [0.01, 0.02, 0.05, 0.1])
def test_rgbd_1280x720_sweep(leaf):
    # key widths from 21 bits (one bin per unit) to 31 bits (units of 2^7 bins)
    check(synth.rgbd_frame(1280, 720, seed=0, cx=639.5, cy=359.5), leaf)


@pytest.mark.parametrize("n", [1, 2, 3, 31, 255, 256, 257, 1023, 1024, 1025, 4095, 4096, 4097,
                               65537, 200_003])
def test_ragged_sizes(n):
    check(synth.random_cloud(n, seed=300 + n, extent=2.0, nan_frac=0.05), 0.02)


@pytest.mark.parametrize("edge", [1, 3, 15, 16, 17, 255, 1023])
def test_key_widths(edge):
    # per-axis extents of `edge` cells: keys from 0 to 30 bits wide in Morton order
    r = np.random.Generator(np.random.PCG64(edge))
    x = (r.random((40_000, 3)) * edge * 0.02).astype(np.float32)
    x[:3] = [[0, 0, 0], [edge * 0.02 - 1e-4] * 3, [0, edge * 0.02 - 1e-4, 0]]
    check(x, 0.02, np.zeros(3, np.float32))


def test_cells_of_many_points():
    # three voxels of 5000+ points: 64-bit per-key sums in shared memory
    r = np.random.Generator(np.random.PCG64(5))
    x = np.concatenate([0.3 + r.random((6000, 3)) * 0.4, 1.3 + r.random((5000, 3)) * 0.4,
                        r.random((3000, 3)) * 3.0]).astype(np.float32)
    got = check(x, 1.0, np.zeros(3, np.float32))
    assert int(gpu_counts(got.counts).max()) >= 6000


def test_keys_wider_than_32_bits_report_range():
    x = np.array([[0, 0, 0], [30.0, 30.0, 30.0], [1, 2, 3]], np.float32)  # 3000 cells/axis
    with pytest.raises(vg.VGError) as e:
        vg.downsample(cuda(x), 0.01, method="frame")
    assert e.value.status == vg.Status.RANGE


def test_empty_and_invalid_clouds():
    for x in (np.zeros((0, 3), np.float32), np.full((100, 3), np.nan, np.float32)):
        got = vg.downsample(cuda(x), 0.05, method="frame")
        assert got.keys.numel() == 0


def test_posed_frame():
    x = synth.rgbd_frame(640, 480, seed=3)
    rt = np.float32([[0.8, -0.6, 0.0, 0.5], [0.6, 0.8, 0.0, -1.0], [0.0, 0.0, 1.0, 0.2]])
    band = np.float32([0.5, 3.0])
    got = vg.downsample(cuda(x), 0.05, pose=rt, z_limits=band, method="frame")
    assert_decimation_equal(got, oracle.downsample_posed(x, 0.05, rt, band), check_p2v=False)
    same_rows(got, vg.downsample(cuda(x), 0.05, pose=rt, z_limits=band, method="sort_lsd"))


def test_other_calls_take_the_sort_path():
    # several frames, or point_to_voxel: the flag is accepted and the plain sort runs
    frames = [synth.rgbd_frame(320, 240, seed=40 + f) for f in range(3)]
    a = vg.downsample_frames([cuda(f) for f in frames], [0.05] * 3, method="frame")
    b = vg.downsample_frames([cuda(f) for f in frames], [0.05] * 3, method="sort_lsd")
    same_rows(a, b)
    x = frames[0]
    got = vg.downsample(cuda(x), 0.05, method="frame", point_to_voxel=True)
    assert_decimation_equal(got, oracle.downsample(x, 0.05))


def test_one_frame_plan_graph_replays():
    x = cuda(synth.rgbd_frame(640, 480, seed=7))
    n = x.shape[0]
    side = torch.cuda.Stream()
    plan = vg.Plan(1, n, method="frame")
    assert plan.get()["method"] == "frame"
    bb = dict(xyz=x, frame_offsets=torch.tensor([0, n], dtype=torch.int64, device="cuda"),
              n_frames=1, origins=torch.zeros((1, 3), dtype=torch.float32, device="cuda"),
              leaves=torch.full((1,), 0.05, dtype=torch.float32, device="cuda"),
              out_keys=torch.empty(n, dtype=torch.int64, device="cuda"),
              out_centroids=torch.empty((n, 3), dtype=torch.float32, device="cuda"),
              out_counts=torch.empty(n, dtype=torch.int32, device="cuda"),
              out_frame_offsets=torch.zeros(2, dtype=torch.int64, device="cuda"),
              out_error=torch.zeros(1, dtype=torch.int32, device="cuda"))
    ref = vg.downsample(x, 0.05, method="sort_lsd")
    with torch.cuda.stream(side):
        for _ in range(3):  # capture, then replays
            bb["out_keys"].fill_(-1)
            plan.run(**bb, graph=True, stream=side)
    side.synchronize()
    plan.close()
    assert int(bb["out_error"].item()) == 0
    v = int(bb["out_frame_offsets"][1].item())
    assert int(bb["out_frame_offsets"][0].item()) == 0
    assert v == ref.keys.numel()
    assert np.array_equal(gpu_keys(bb["out_keys"][:v]), gpu_keys(ref.keys))
    assert np.array_equal(gpu_counts(bb["out_counts"][:v]), gpu_counts(ref.counts))
    assert np.array_equal(to_np(bb["out_centroids"][:v]), to_np(ref.centroids))


def test_one_launch_capacity():
    cap = vg.frame_one_launch_points()
    assert 1920 * 1080 <= cap <= 2 ** 21  # one block of 1024 threads an SM, 14 points a thread
    assert vg.frame_one_launch_points(posed=True) >= 640 * 480


def test_full_hd_one_launch():
    check(synth.rgbd_frame(1920, 1080, seed=12, cx=959.5, cy=539.5), 0.02)


@pytest.mark.parametrize("w,h", [(2304, 1296), (2560, 1440)])
def test_frames_beyond_one_launch(w, h):
    # above the one-launch capacity the bin grouping (five kernels) takes the frame
    if w * h <= vg.frame_one_launch_points():
        pytest.skip("this device's one-launch grid holds the frame")
    check(synth.rgbd_frame(w, h, seed=11, cx=w / 2 - 0.5, cy=h / 2 - 0.5), 0.02)


@pytest.mark.parametrize("leaf", [0.005, 0.01])
def test_wide_keys_one_launch(leaf):
    # 24-bit keys (the bitmap the kernel clears before the extents) and 27-bit keys
    # (bitmaps of the occupied blocks of 2^9 keys, numbered first)
    x = synth.rgbd_frame(640, 480, seed=21)
    got = check(x, leaf)
    assert got.keys.numel() > 0


def test_repeated_calls_same_buffers():
    # the grid-barrier counter and scan words are reset every call: calls in a row agree
    x = cuda(synth.rgbd_frame(640, 480, seed=8))
    b = vg.alloc_buffers(x.shape[0], "cuda", flags=vg.method_flag("frame"))
    ref = vg.downsample(x, 0.05, method="sort_lsd")
    for leaf in (0.05, 0.004, 0.05):
        vg.downsample_into(x, leaf, b, origin_from_min=True, method="frame")
        assert int(b.error.item()) == 0
    v = int(b.num_voxels.item())
    assert v == ref.keys.numel()
    assert np.array_equal(gpu_keys(b.keys[:v]), gpu_keys(ref.keys))
    assert np.array_equal(to_np(b.centroids[:v]), to_np(ref.centroids))


def test_bad_offsets_one_frame():
    xyz = cuda(synth.random_cloud(1000, seed=1))
    with pytest.raises(vg.VGError) as e:
        vg.downsample_frames((xyz, [0, 999]), [0.1], method="frame")
    assert e.value.status == vg.Status.INVALID_ARG
    # the next call with the same method is unaffected
    x = synth.random_cloud(1000, seed=1)
    check(x, 0.1)


@pytest.mark.parametrize("cells,bits", [((511, 511, 255), 26), ((511, 511, 511), 27),
                                        ((1023, 1023, 511), 29)])
def test_bitmap_widths(cells, bits):
    # 26-bit keys: the widest single key bitmap (its words past 2^19 cleared after the
    # extents); 27 and 29 bits: bitmaps of the occupied blocks of 2^9 keys
    r = np.random.Generator(np.random.PCG64(bits))
    ext = np.float32(cells) * np.float32(0.02)
    x = (r.random((60_000, 3)) * ext).astype(np.float32)
    x[0] = ext - np.float32(1e-3)
    x[1] = 0.0
    got = check(x, 0.02, np.zeros(3, np.float32))
    assert int(gpu_keys(got.keys).max()).bit_length() == bits


def test_grid_barrier_wait_times_out():
    # the one-launch kernel's grid barrier: a wait nobody completes gives up and reports
    scratch = torch.zeros(4, dtype=torch.int32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = vg.lib().vg_debug_grid_barrier_timeout(vg._ptr(scratch), 1000, vg._ptr(err), None)
    assert st == 0
    torch.cuda.synchronize()
    assert int(err.item()) == vg.Status.TIMEOUT
    assert int(scratch[0].item()) == 2  # both blocks arrived
    # the context is usable afterwards
    check(synth.random_cloud(5000, seed=77), 0.05)


def test_capacity_short_of_the_voxels():
    # 100 output rows for 11,489 voxels: the rows that fit are written, V is counted in
    # full, and the call reports the shortfall
    x = cuda(synth.rgbd_frame(640, 480, seed=0))
    b = vg.alloc_buffers(x.shape[0], "cuda", flags=vg.method_flag("frame"))
    vg.downsample_into(x, 0.05, b, origin_from_min=True, method="frame", cap=100)
    torch.cuda.synchronize()
    assert int(b.error.item()) == vg.Status.CAPACITY
    ref = vg.downsample(x, 0.05, method="sort_lsd")
    assert int(b.num_voxels.item()) == ref.keys.numel()
    assert np.array_equal(gpu_keys(b.keys[:100]), gpu_keys(ref.keys[:100]))
    assert np.array_equal(to_np(b.centroids[:100]), to_np(ref.centroids[:100]))
