"""Batched frames (vg_downsample_frames / vg_downsample_batch): every frame against the
oracle, bit-equality with solo calls, CUDA-graph replay, the autotuner, bad offsets."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_11084_gb300 import synth, vg
from tests._parity import assert_decimation_equal, gpu_counts, gpu_keys, to_np

pytestmark = pytest.mark.gpu


def small_batch(seed=0, frames=9):
    rng = np.random.Generator(np.random.PCG64(seed))
    out, leaves = [], []
    for f in range(frames):
        full = synth.rgbd_frame(160, 120, seed=300 + f)
        n = int(rng.integers(0, full.shape[0]))
        if f == 3:
            n = 0  # an empty frame
        keep = np.sort(rng.choice(full.shape[0], n, replace=False))
        out.append(np.ascontiguousarray(full[keep]))
        leaves.append(float(rng.choice([0.02, 0.05, 0.1])))
    if frames > 5:
        out[5][:] = np.nan  # an all-invalid frame
    return out, np.asarray(leaves, np.float32)


def check_frames(res, frames, leaves):
    for f, x in enumerate(frames):
        ref = oracle.downsample(x, float(leaves[f]))
        d = res.frame(f)
        assert_decimation_equal(d, ref, check_p2v=False)


@pytest.mark.parametrize("method", ["sort", "hash"])
def test_frames_against_oracle(method):
    frames, leaves = small_batch()
    res = vg.downsample_frames([torch.from_numpy(x).cuda() for x in frames], leaves,
                               method=method, point_to_voxel=True)
    check_frames(res, frames, leaves)
    # point_to_voxel: global rows = frame offset + the frame's own oracle rows
    p2v = to_np(res.point_to_voxel)
    pos = 0
    for f, x in enumerate(frames):
        ref = oracle.downsample(x, float(leaves[f]))
        want = np.where(ref.point_to_voxel >= 0, ref.point_to_voxel + res.offsets[f], -1)
        assert np.array_equal(p2v[pos:pos + len(x)], want)
        pos += len(x)


def test_frames_bit_identical_to_solo_calls():
    frames, leaves = small_batch(seed=1)
    res = vg.downsample_frames([torch.from_numpy(x).cuda() for x in frames], leaves)
    for f, x in enumerate(frames):
        solo = vg.downsample(torch.from_numpy(x).cuda(), float(leaves[f]))
        d = res.frame(f)
        assert torch.equal(d.keys, solo.keys) and torch.equal(d.counts, solo.counts)
        assert torch.equal(d.centroids.view(torch.int32), solo.centroids.view(torch.int32))


def test_given_origins():
    frames, leaves = small_batch(seed=2, frames=4)
    origins = np.array([[-4.0, -3.0, 0.0]] * 4, np.float32)
    res = vg.downsample_frames([torch.from_numpy(x).cuda() for x in frames], leaves, origins)
    for f, x in enumerate(frames):
        ref = oracle.downsample(x, float(leaves[f]), origins[f])
        d = res.frame(f)
        assert np.array_equal(gpu_keys(d.keys), ref.keys)
        assert np.array_equal(gpu_counts(d.counts), ref.counts)


def test_bad_frame_offsets_are_reported():
    xyz = torch.from_numpy(synth.random_cloud(1000, 1)).cuda()
    with pytest.raises(vg.VGError) as e:
        vg.downsample_frames((xyz, [0, 600, 500, 1000]), [0.1, 0.1, 0.1])
    assert e.value.status == vg.Status.INVALID_ARG
    with pytest.raises(vg.VGError):
        vg.downsample_frames((xyz, [0, 400, 999]), [0.1, 0.1])


def _plan_buffers(frames, leaves):
    xyz = torch.cat([torch.from_numpy(x) for x in frames]).cuda().contiguous()
    offs = np.cumsum([0] + [len(x) for x in frames])
    F = len(frames)
    n = xyz.shape[0]
    b = dict(xyz=xyz, frame_offsets=torch.tensor(offs, dtype=torch.int64, device="cuda"),
             n_frames=F, origins=torch.zeros((F, 3), dtype=torch.float32, device="cuda"),
             leaves=torch.from_numpy(np.asarray(leaves, np.float32)).cuda(),
             out_keys=torch.empty(n, dtype=torch.int64, device="cuda"),
             out_centroids=torch.empty((n, 3), dtype=torch.float32, device="cuda"),
             out_counts=torch.empty(n, dtype=torch.int32, device="cuda"),
             out_frame_offsets=torch.zeros(F + 1, dtype=torch.int64, device="cuda"),
             out_error=torch.zeros(1, dtype=torch.int32, device="cuda"))
    return b


def test_plan_graph_replay_and_tuner():
    frames, leaves = small_batch(seed=4, frames=12)
    ref = vg.downsample_frames([torch.from_numpy(x).cuda() for x in frames], leaves)
    b = _plan_buffers(frames, leaves)
    plan = vg.Plan(16, b["xyz"].shape[0])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        times = plan.tune(**b, reps=2, stream=s)
        assert len(times) == 12
        assert all(t > 0 for k, t in times.items() if not k.startswith("frame"))
        assert all(times[f"frame@{g}"] == -1 for g in (4, 8, 16))  # several frames: not timed
        for _ in range(3):  # graph replays
            plan.run(**b, stream=s)
        s.synchronize()
    assert int(b["out_error"].item()) == 0
    offs = b["out_frame_offsets"].cpu().tolist()
    assert offs == ref.offsets
    v = offs[-1]
    assert torch.equal(b["out_keys"][:v], ref.keys)
    assert torch.equal(b["out_counts"][:v], ref.counts)
    assert torch.equal(b["out_centroids"][:v].view(torch.int32), ref.centroids.view(torch.int32))
    for m in ("auto", "sort", "sort_lsd", "frame", "hash"):
        plan.configure(m, 8)
        assert plan.get()["method"] == m
        with torch.cuda.stream(s):
            plan.run(**b, stream=s, graph=False)
            s.synchronize()
        assert torch.equal(b["out_keys"][:v], ref.keys)
    plan.close()


def test_one_frame_tuning_times_the_bin_grouping():
    frame = synth.rgbd_frame(640, 480, seed=12)
    b = _plan_buffers([frame], [0.05])
    plan = vg.Plan(1, b["xyz"].shape[0])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        times = plan.tune(**b, reps=2, stream=s)
    assert all(t > 0 for t in times.values())
    best = min(times, key=times.get).split("@")[0]
    assert plan.get()["method"] == best
    plan.close()
    # keys wider than 32 bits: the bin grouping records an error, so it is not a candidate
    wide = np.array([[0, 0, 0], [30.0, 30.0, 30.0], [1, 2, 3]] * 100, np.float32)
    b = _plan_buffers([wide], [0.01])
    plan = vg.Plan(1, b["xyz"].shape[0])
    with torch.cuda.stream(s):
        times = plan.tune(**b, reps=1, stream=s)
        s.synchronize()
    assert all(times[f"frame@{g}"] == -1 for g in (4, 8, 16))
    assert plan.get()["method"] != "frame"
    assert int(b["out_error"].item()) == 0
    plan.close()


def test_plan_tuning_persists(tmp_path):
    frames, leaves = small_batch(seed=5, frames=6)
    b = _plan_buffers(frames, leaves)
    plan = vg.Plan(8, b["xyz"].shape[0])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.tune(**b, reps=1, stream=s)
    chosen = plan.get()
    path = str(tmp_path / "tuning.json")
    plan.save_tuning(path, workload="small batch")
    other = vg.Plan(8, b["xyz"].shape[0])
    other.configure("hash" if chosen["method"] == "sort" else "sort", 4)
    rec = other.load_tuning(path)
    assert other.get()["method"] == chosen["method"] == rec["method"]
    assert other.get()["grid_per_sm"] == chosen["grid_per_sm"]
    with pytest.raises(ValueError):
        vg.Plan(9, b["xyz"].shape[0]).load_tuning(path)
    plan.close()
    other.close()


def test_batch_64_frames_full_size():
    """The 64-frame uneven batch (20k-921k points per 1280x720 frame, leaf per frame from
    {0.02, 0.05, 0.1}): every frame bit-equal to its solo call, four sampled frames
    against the oracle."""
    spec = synth.batch_frames(64, seed=1)
    dev = [torch.from_numpy(x).cuda() for x in spec.frames]
    res = vg.downsample_frames(dev, spec.leaves)
    for f in range(64):
        solo = vg.downsample(dev[f], float(spec.leaves[f]))
        d = res.frame(f)
        assert torch.equal(d.keys, solo.keys) and torch.equal(d.counts, solo.counts)
        assert torch.equal(d.centroids.view(torch.int32), solo.centroids.view(torch.int32))
    for f in (0, 17, 40, 63):
        ref = oracle.downsample(spec.frames[f], float(spec.leaves[f]))
        assert_decimation_equal(res.frame(f), ref, check_p2v=False)


def test_bounded_wait_times_out():
    scratch = torch.zeros(4, dtype=torch.int32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = vg.lib().vg_debug_wait_timeout(vg._ptr(scratch), 1000, vg._ptr(err), None)
    assert st == 0
    torch.cuda.synchronize()
    assert int(err.item()) == vg.Status.TIMEOUT
