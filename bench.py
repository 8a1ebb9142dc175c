"""Benchmark of voxel-grid decimation on GB300 (one JSON line on stdout).

Workload: the fused map cloud -- 50,000,000 FP32 points (70 % on planes/box surfaces in a
40 x 40 x 10 m volume with 5 mm noise, 30 % uniform clutter, 2 % NaN, globally
shuffled), origin = cloud minimum, leaf 0.02 m.  One step = one vg_downsample call over
the whole cloud (origin, keys, radix sort, segmented reduction + compaction).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (under torchrun) runs one independent replica per GPU (the path has no exchange
step) and reports the points of all ranks over the slowest rank's time.
--impl reference times the CPU oracle (FP64 std::map, one core) on a bounded sample of
the same workload, as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_POINTS = 50_000_000
LEAF = 0.02
WORKLOAD = "fused map cloud, 50M xyz f32 points, 40x40x10 m, leaf 0.02 m, origin = cloud min"
REFERENCE_SAMPLE = 250_000    # --impl reference: points per step


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="vg", choices=["vg", "reference"])
    p.add_argument("--n", type=int, default=N_POINTS)
    p.add_argument("--leaf", type=float, default=LEAF)
    p.add_argument("--method", default="auto", choices=["auto", "sort", "sort_lsd", "hash"],
                   help="grouping of the timed step: the library's choice (the bucket "
                        "grouping for a cloud this large), the sort with bucket grouping, the "
                        "global LSD radix sort, or the hash path")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the other configurations (single frame, batch, pyramid, "
                        "backward, leaf 0.1 m, serving)")
    p.add_argument("--serve-seconds", type=float, default=10.0)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device) -> float:
    """The slowest replica's value (the job ends when its last rank does); x on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device) -> float:
    """Total over the replicas (points processed by the whole job)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.stamped = []

    def _read(self):
        for line in self.proc.stdout:
            if line.strip():
                self.stamped.append((time.perf_counter(), line))

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        if self.proc is not None:
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
            t_wait = time.perf_counter() + 5.0  # the sampler is running before timing starts
            while not self.stamped and time.perf_counter() < t_wait and self.proc.poll() is None:
                time.sleep(0.01)
        self.t0 = time.perf_counter()
        return self

    def __exit__(self, *a):
        self.t1 = time.perf_counter()
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
            self.reader.join(timeout=5)
            inside = [l for ts, l in self.stamped if self.t0 <= ts <= self.t1 + 0.05]
            self.lines = inside or [l for _, l in self.stamped[-1:]]

    def summary(self):
        if not getattr(self, "lines", None):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# the sources of the kernels the bench step launches (their traffic is profiled)
STEP_KERNEL_SOURCES = ("vg_device.cuh", "vg_internal.h", "vg_keys.cu", "vg_msd.cu",
                       "vg_reduce.cu", "vg_rows.cuh", "vg_sort.cu", "vg_stream.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2102_11084_gb300", "csrc")
    for f in STEP_KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(units: dict):
    """DRAM bytes of one step from the committed ncu summary (per kernel: bytes per unit x
    the units of this run), if it was taken on the current sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    total = 0.0
    for name, k in d.get("kernels", {}).items():
        total += float(k["bytes_per_unit"]) * float(units[k["unit"]]) * float(k.get("launches", 1))
    return total


# --------------------------------------------------------------------------------------
def _time_ms(fn, reps, warmup=3, stream=None):
    """Mean device ms of fn() over `reps` calls (CUDA events on the launching stream)."""
    import torch
    s = stream or torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        fn()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def extra_measurements(args, dev, peak):
    """The other configurations of the workload set, each timed on the device."""
    import torch
    from paper_2102_11084_gb300 import serve, synth, vg
    out = {}
    stream = torch.cuda.current_stream(dev)

    # 640x480 RGB-D frame, leaf 0.05 m: one plain call per grouping (host issue is well
    # under the device time, so back-to-back calls measure the device), and the one-frame
    # plan (CUDA-graph replay)
    frame = synth.rgbd_frame(640, 480, seed=0)
    x = torch.from_numpy(frame).to(dev)
    n = x.shape[0]
    r = {}
    for m in ("auto", "frame", "sort", "sort_lsd", "hash"):
        buf = vg.alloc_buffers(n, dev, flags=vg.method_flag(m))
        ms = _time_ms(lambda: vg.downsample_into(x, 0.05, buf, origin_from_min=True, method=m), 200)
        if int(buf.error.item()):
            raise vg.VGError(int(buf.error.item()), "640x480 " + m)
        v = int(buf.num_voxels.item())
        r[m] = {"ms": ms, "points_per_s": n / (ms / 1e3),
                "roofline_frac": (12.0 * n + 16.0 * v) / (ms / 1e3) / 1e9 / peak}
    side1 = torch.cuda.Stream(dev)
    fb = dict(xyz=x, frame_offsets=torch.tensor([0, n], dtype=torch.int64, device=dev),
              n_frames=1, origins=torch.zeros((1, 3), dtype=torch.float32, device=dev),
              leaves=torch.full((1,), 0.05, dtype=torch.float32, device=dev),
              out_keys=torch.empty(n, dtype=torch.int64, device=dev),
              out_centroids=torch.empty((n, 3), dtype=torch.float32, device=dev),
              out_counts=torch.empty(n, dtype=torch.int32, device=dev),
              out_frame_offsets=torch.zeros(2, dtype=torch.int64, device=dev),
              out_error=torch.zeros(1, dtype=torch.int32, device=dev))
    for m in ("frame", "sort_lsd"):
        plan1 = vg.Plan(1, n, method=m)
        with torch.cuda.stream(side1):
            ms = _time_ms(lambda: plan1.run(**fb, graph=True, stream=side1), 200, stream=side1)
        plan1.close()
        r["plan_graph_" + m] = {"ms": ms, "points_per_s": n / (ms / 1e3),
                                "roofline_frac": (12.0 * n + 16.0 * v) / (ms / 1e3) / 1e9 / peak}
    r["voxels"] = v
    r["auto_choice"] = ("sort_lsd (radix sort: fewer than 2^22 points; the one-launch frame "
                        "grouping needs 32-bit keys, known only on the device)")
    out["rgbd_640x480_leaf0.05"] = r

    # 64 frames of uneven size: 64 plain calls vs one batched call (plan, tuned, graph)
    spec = synth.batch_frames(64, seed=1)
    frames = [torch.from_numpy(f).to(dev) for f in spec.frames]
    sizes = [f.shape[0] for f in frames]
    total = int(sum(sizes))
    bufs = [vg.alloc_buffers(k, dev) for k in sizes]

    def per_frame():
        for f, b, lf in zip(frames, bufs, spec.leaves):
            vg.downsample_into(f, float(lf), b, origin_from_min=True)
    ms_per_frame = _time_ms(per_frame, 10)
    xyz = torch.cat(frames).contiguous()
    offs = torch.tensor([0] + list(np.cumsum(sizes)), dtype=torch.int64, device=dev)
    F = len(frames)
    bb = dict(xyz=xyz, frame_offsets=offs, n_frames=F,
              origins=torch.zeros((F, 3), dtype=torch.float32, device=dev),
              leaves=torch.from_numpy(spec.leaves).to(dev),
              out_keys=torch.empty(total, dtype=torch.int64, device=dev),
              out_centroids=torch.empty((total, 3), dtype=torch.float32, device=dev),
              out_counts=torch.empty(total, dtype=torch.int32, device=dev),
              out_frame_offsets=torch.zeros(F + 1, dtype=torch.int64, device=dev),
              out_error=torch.zeros(1, dtype=torch.int32, device=dev))
    side = torch.cuda.Stream(dev)
    plan = vg.Plan(F, total)
    with torch.cuda.stream(side):
        tuned = plan.tune(**bb, reps=5, stream=side)
        ms_batched = _time_ms(lambda: plan.run(**bb, stream=side), 20, stream=side)
    chosen = plan.get()
    plan.close()
    out["batch_64_frames"] = {
        "points": total, "per_frame_calls_ms": ms_per_frame, "batched_graph_ms": ms_batched,
        "speedup": ms_per_frame / ms_batched, "batched_points_per_s": total / (ms_batched / 1e3),
        "tuned": {"method": chosen["method"], "grid_per_sm": chosen["grid_per_sm"],
                  "candidates_ms": tuned}}

    # the same 64 frames, posed: each camera cloud taken into the map frame and cut to the
    # height band in the same call (vg_downsample_frames_posed) vs the plain call
    poses, bands = synth.sensor_poses(F, seed=2)
    pz = torch.from_numpy(poses.reshape(F, 12)).to(dev)
    zl = torch.from_numpy(bands).to(dev)
    wsf = torch.empty(int(vg.lib().vg_batch_workspace_bytes(total, F, vg.METHOD_SORT)),
                      dtype=torch.uint8, device=dev)
    fargs = dict(xyz=xyz, frame_offsets=offs, n_frames=F, origins=bb["origins"],
                 leaves=bb["leaves"], out_keys=bb["out_keys"], out_centroids=bb["out_centroids"],
                 out_counts=bb["out_counts"], out_frame_offsets=bb["out_frame_offsets"],
                 out_error=bb["out_error"], workspace=wsf)
    ms_plain = _time_ms(lambda: vg.frames_into(**fargs), 20)
    v_plain = int(bb["out_frame_offsets"][F].item())
    ms_posed = _time_ms(lambda: vg.frames_into(**fargs, poses=pz, z_limits=zl), 20)
    if int(bb["out_error"].item()):
        raise vg.VGError(int(bb["out_error"].item()), "posed batch")
    out["batch_64_frames_posed"] = {
        "points": total, "plain_call_ms": ms_plain, "posed_call_ms": ms_posed,
        "posed_points_per_s": total / (ms_posed / 1e3), "overhead": ms_posed / ms_plain - 1.0,
        "voxels_plain": v_plain, "voxels_posed": int(bb["out_frame_offsets"][F].item()),
        "band_m": [float(b) for b in bands[0]]}

    # persistent voxel map: the 64 posed frames merged into one map (one insert call after
    # a clear), then the whole map extracted in key order
    mp = vg.VoxelMap(4_000_000, (-20.0, -20.0, -5.0), 0.05, device=dev)
    sp = vg._stream_ptr(None)

    def map_insert():
        vg.lib().vg_map_clear(mp._h, sp)
        vg.lib().vg_map_insert(mp._h, vg._ptr(xyz), total, vg._ptr(offs), F, vg._ptr(pz),
                               vg._ptr(zl), vg._ptr(mp.error), sp)
    ms_ins = _time_ms(map_insert, 20)
    mk = torch.empty(8_000_000, dtype=torch.int64, device=dev)
    mc = torch.empty((8_000_000, 3), dtype=torch.float32, device=dev)
    mn = torch.empty(8_000_000, dtype=torch.int32, device=dev)
    mv = torch.zeros(1, dtype=torch.int64, device=dev)
    ms_ext = _time_ms(lambda: vg.lib().vg_map_extract(
        mp._h, vg._ptr(mk), vg._ptr(mc), vg._ptr(mn), mk.shape[0], vg._ptr(mv),
        vg._ptr(mp.error), sp), 20)
    if int(mp.error.item()):
        raise vg.VGError(int(mp.error.item()), "voxel map")
    out["voxel_map_64_posed_frames"] = {
        "points": total, "insert_ms": ms_ins, "insert_points_per_s": total / (ms_ins / 1e3),
        "extract_ms": ms_ext, "voxels": int(mv.item()), "leaf_m": 0.05, "slots": 8_388_608}
    mp.close()
    del frames, bufs, xyz, bb, fargs, wsf, mk, mc, mn

    # 1280x720 frame: 4-level pyramid from 0.01 m, and the leaf sweep
    hd = torch.from_numpy(synth.rgbd_frame(1280, 720, seed=0, cx=639.5, cy=359.5)).to(dev)
    out["pyramid_1280x720_4_levels_ms"] = _time_ms(lambda: vg.pyramid(hd, 0.01, 4), 20)
    sweep = {}
    nhd = hd.shape[0]
    for m in ("auto", "frame"):
        hb = vg.alloc_buffers(nhd, dev, flags=vg.method_flag(m))
        for lf in (0.01, 0.02, 0.05, 0.1):
            ms = _time_ms(lambda: vg.downsample_into(hd, lf, hb, origin_from_min=True, method=m),
                          50)
            if int(hb.error.item()):
                raise vg.VGError(int(hb.error.item()), "1280x720 " + m)
            vh = int(hb.num_voxels.item())
            sweep.setdefault(str(lf), {"voxels": vh})[m] = {
                "ms": ms, "points_per_s": nhd / (ms / 1e3),
                "roofline_frac": (12.0 * nhd + 16.0 * vh) / (ms / 1e3) / 1e9 / peak}
    out["rgbd_1280x720_sweep"] = sweep

    # voxel extras on the same frame at 0.02 m: RGB means per voxel and/or min 2 points
    nh = hd.shape[0]
    rgb = torch.randint(0, 256, (nh, 3), dtype=torch.uint8, device=dev,
                        generator=torch.Generator(device=dev).manual_seed(7))
    one = torch.tensor([0, nh], dtype=torch.int64, device=dev)
    lf = torch.tensor([0.02], dtype=torch.float32, device=dev)
    og = torch.zeros((1, 3), dtype=torch.float32, device=dev)
    o_at = torch.empty((nh, 3), dtype=torch.float32, device=dev)
    o_off = torch.zeros(2, dtype=torch.int64, device=dev)
    ext = {}
    for name, kw in (("plain", {}), ("rgb_means", {"attrs": rgb, "out_attrs": o_at}),
                     ("min_count_2", {"min_count": 2}),
                     ("rgb_means_min_count_2", {"attrs": rgb, "out_attrs": o_at,
                                                "min_count": 2})):
        exs = vg.extras(kw.get("attrs"), kw.get("out_attrs"), kw.get("min_count", 1))
        wsx = torch.empty(max(vg.ex_workspace_bytes(nh, 1, vg.METHOD_SORT, exs), 256),
                          dtype=torch.uint8, device=dev)
        ms = _time_ms(lambda: vg.frames_into(hd, one, 1, og, lf, hb.keys, hb.centroids,
                                             hb.counts, o_off, hb.error, wsx, **kw), 50)
        ext[name] = {"ms": ms, "points_per_s": nh / (ms / 1e3), "voxels": int(o_off[1].item())}
    out["rgbd_1280x720_leaf0.02_extras"] = ext

    # the paper's own neighbour-count thinning loop on the 640x480 frame: cell = radius
    # 0.05 m, threshold 20, batches of 1000 (host-synchronised once per pass and per
    # select round, so timed on the host clock around whole calls)
    pr = torch.from_numpy(np.random.Generator(np.random.PCG64(5)).permutation(n)
                          .astype(np.uint32).view(np.int32)).to(dev)
    vg.thin(x, 0.05, 20, pr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 5
    for _ in range(reps):
        th = vg.thin(x, 0.05, 20, pr)
    torch.cuda.synchronize()
    ms_thin = (time.perf_counter() - t0) / reps * 1e3
    out["thin_640x480_cell0.05_t20_b1000"] = {"ms": ms_thin, "passes": th.passes,
                                               "kept": th.num_kept,
                                               "ms_per_pass": ms_thin / max(th.passes, 1)}

    # backward of the mean squared centroid loss, 307,200 points, leaf 0.05 m
    res = vg.downsample(x, 0.05, point_to_voxel=True)
    g = torch.randn_like(res.centroids)
    out["backward_640x480_ms"] = _time_ms(
        lambda: vg.backward(g, res.counts, res.point_to_voxel, check=False), 200)

    # serving: 16 sensor streams x 30 Hz Poisson arrivals of 640x480 frames, leaf 0.05 m;
    # camera frames, so the frame method (a batch of one frame in one launch)
    pool = [synth.rgbd_frame(640, 480, seed=3000 + k) for k in range(64)]
    trace = synth.serving_trace(16, 30.0, args.serve_seconds, len(pool), seed=5)
    srv = serve.Server(max_points=16 * 307_200, max_frames=16, n_slots=3, record_timeline=True,
                       method="frame")
    results, wall = serve.replay(srv, trace, pool, 0.05)
    tl = srv.timeline()
    srv.close()
    st = serve.latency_stats(results)
    st["copy_overlap"] = serve.copy_overlap(tl)
    st["points_per_s"] = len(results) * 307_200 / wall
    st["wall_s"] = wall
    st["batches"] = srv.batches
    sat_trace = [r._replace(arrival_s=0.0) for r in trace[:2000]]
    srv = serve.Server(max_points=16 * 307_200, max_frames=16, n_slots=3, record_timeline=True,
                       method="frame")
    sat, sat_wall = serve.replay(srv, sat_trace, pool, 0.05, realtime=False)
    sat_tl = srv.timeline()
    srv.close()
    st["saturation_points_per_s"] = len(sat) * 307_200 / sat_wall
    st["saturation_p99_ms"] = serve.latency_stats(sat)["p99_ms"]
    st["saturation_copy_overlap"] = serve.copy_overlap(sat_tl)
    st["copy_overlap_definition"] = ("copy time (pinned host <-> device, in and out) that ran "
                                     "while another batch was decimated, over all copy time; "
                                     "CUDA event timestamps")
    st["method"] = "frame"
    out["serving_16x30Hz_640x480"] = st
    return out


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on bounded samples of the same workload."""
    if rank != 0:
        return
    import oracle
    from paper_2102_11084_gb300 import synth
    xyz = synth.fused_map(args.n, seed=0)
    # bounded work: the whole run stays near a minute of CPU time whatever --steps is
    per_step = max(20_000, REFERENCE_SAMPLE * 50 // max(args.steps + args.warmup, 50))
    sample = np.ascontiguousarray(xyz[:per_step])
    for _ in range(args.warmup):
        oracle.downsample(sample, args.leaf)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.downsample(sample, args.leaf)
        times.append(time.perf_counter() - t0)
    ms = 1000 * statistics.mean(times)
    value = sample.shape[0] / (ms / 1000)
    sample_desc = f"first {sample.shape[0]} points of the workload cloud per step, 1 thread"
    print(json.dumps({
        "impl": "reference", "metric": "points/s", "value": value, "unit": "points/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "leaf_m": args.leaf},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


ORACLE_CLOUD_SNIPPET = (
    "import sys, time, numpy as np\n"
    "sys.path.insert(0, sys.argv[1])\n"
    "import oracle\n"
    "x = np.load(sys.argv[2], mmap_mode='r')\n"
    "x = np.ascontiguousarray(x)\n"
    "t0 = time.perf_counter()\n"
    "oracle.downsample(x, float(sys.argv[3]))\n"
    "print(time.perf_counter() - t0)\n")


class OracleTimer:
    """The single-threaded oracle timed on the whole workload cloud, once, in a separate
    process (fork + exec, started before this process's timed GPU work and collected at
    the end), so the CPU run overlaps the GPU measurements."""

    def __init__(self, xyz, leaf):
        import tempfile
        self.tmp = tempfile.NamedTemporaryFile(suffix=".npy", delete=False)
        self.tmp.close()
        np.save(self.tmp.name, xyz)
        self.n = xyz.shape[0]
        self.proc = subprocess.Popen([sys.executable, "-c", ORACLE_CLOUD_SNIPPET, ROOT,
                                      self.tmp.name, repr(float(leaf))],
                                     stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)

    def result(self):
        try:
            out, errs = self.proc.communicate(timeout=1800)
            dt = float(out.strip().splitlines()[-1])
        except (subprocess.TimeoutExpired, ValueError, IndexError):
            self.proc.kill()
            return None
        finally:
            os.unlink(self.tmp.name)
        return dt


def cpu_baseline(oracle_timer, frame_xyz):
    """cpu_baseline: the oracle (std::map, FP64, one thread) on the whole workload cloud,
    once, plus the 640x480 frame at leaf 0.05 m with 10 repetitions."""
    import oracle
    dt = oracle_timer.result() if oracle_timer else None
    reps = 10
    oracle.downsample(frame_xyz, 0.05)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.downsample(frame_xyz, 0.05)
    dt_frame = (time.perf_counter() - t0) / reps
    out = {"unit": "points/s", "cores": 1, "kind": "oracle",
           "host_cores_available": os.cpu_count(),
           "rgbd_640x480_leaf0.05": {"ms": dt_frame * 1e3,
                                     "points_per_s": frame_xyz.shape[0] / dt_frame,
                                     "reps": reps}}
    if dt is not None:
        out["value"] = oracle_timer.n / dt
        out["sample"] = (f"the whole workload cloud ({oracle_timer.n} points, same leaf, "
                         f"origin = cloud min), once: {dt:.1f} s on one core; single-threaded "
                         f"std::map FP64 oracle")
    else:
        out["value"] = None
        out["sample"] = "the whole-cloud oracle run did not finish"
    return out


def run_vg(args, rank, world, local):
    import torch
    import torch.distributed as dist
    from paper_2102_11084_gb300 import synth, vg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl")
    xyz_np = synth.fused_map(args.n, seed=rank)
    n = xyz_np.shape[0]
    xyz_host = torch.from_numpy(xyz_np).pin_memory()
    xyz = xyz_host.to(dev)
    buf = vg.alloc_buffers(n, dev)
    stream = torch.cuda.current_stream(dev)

    # the single-threaded oracle on the whole cloud, in another process while the GPU works
    oracle_timer = (OracleTimer(xyz_np, args.leaf)
                    if rank == 0 and not args.no_cpu_baseline else None)

    # stage events (profiling hook of the C ABI): one set per timed step.  Sort path:
    # extent/origin, keys, the bucket grouping's first partition pass, second partition
    # pass and bucket kernel, 8 radix passes (the needed ones do work; none with the bucket
    # grouping), the segmented reduction (returns at once with the bucket grouping)
    n_stages = 14
    import ctypes

    def call():
        vg.downsample_into(xyz, args.leaf, buf, origin_from_min=True, method=args.method,
                           stream=stream)

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    err = int(buf.error.item())
    if err:
        raise vg.VGError(err, "warm-up")

    ev_sets = [[torch.cuda.Event(enable_timing=True) for _ in range(n_stages + 1)]
               for _ in range(args.steps)]
    # create the underlying CUDA events
    for s in ev_sets:
        for e in s:
            e.record(stream)
    torch.cuda.synchronize()
    arrs = [(ctypes.c_void_p * (n_stages + 1))(*[ctypes.c_void_p(e.cuda_event) for e in s])
            for s in ev_sets]

    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        for k in range(args.steps):
            vg.lib().vg_set_stage_events(arrs[k], n_stages + 1)
            call()
        stop.record(stream)
        torch.cuda.synchronize()
    vg.lib().vg_set_stage_events(None, 0)
    ms = start.elapsed_time(stop) / args.steps
    ms = max_over_ranks(ms, dev)
    total_points = sum_over_ranks(n, dev)
    err = int(buf.error.item())
    if err:
        raise vg.VGError(err, "timed steps")
    V = int(buf.num_voxels.item())
    nvalid = int(np.isfinite(xyz_np).all(axis=1).sum())

    # per-stage device times (ms, mean over steps)
    stage_names = (["origin", "keys", "partition1", "partition2", "bucket"] +
                   [f"sort_pass{p}" for p in range(8)] + ["segreduce"])
    stage_ms = np.zeros(n_stages)
    for s in ev_sets:
        for i in range(n_stages):
            stage_ms[i] += s[i].elapsed_time(s[i + 1])
    stage_ms /= args.steps
    st_ms = dict(zip(stage_names, (float(v) for v in stage_ms)))
    bucketed = st_ms["bucket"] > 0.02  # the bucket grouping ran (else the global radix sort)
    passes = int((stage_ms[5:13] > 0.02).sum())
    narrow = int(buf.keys[V - 1].item()).bit_length() <= 32 if V else True
    # algorithmic bytes of each kernel group per launch: narrow entries are a 4 B key and an
    # 8 B packed offset; every output row is an 8 B key, a 12 B centroid and a 4 B count
    algo = {
        "origin": 12.0 * n,
        "keys": 12.0 * n + 12.0 * n,
        "partition1": 4.0 * n + 8.0 * nvalid + 12.0 * nvalid,
        "partition2": 4.0 * nvalid + 24.0 * nvalid,
        "bucket": 12.0 * nvalid + 24.0 * V,
        "sort_pass": 24.0 * nvalid,
        "segreduce": ((4.0 + 12.0) if narrow else (8.0 + 24.0)) * nvalid + 24.0 * V,
    }
    kern = {"origin": (st_ms["origin"], 1), "keys": (st_ms["keys"], 1)}
    if bucketed:
        kern.update({"partition1": (st_ms["partition1"], 1),
                     "partition2": (st_ms["partition2"], 1), "bucket": (st_ms["bucket"], 1)})
    else:
        kern.update({"sort_pass": (float(stage_ms[5:5 + max(passes, 1)].mean()), max(passes, 1)),
                     "segreduce": (st_ms["segreduce"], 1)})
    dom = max(kern, key=lambda k: kern[k][0] * kern[k][1])
    peaks, peak_src = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    d_ms = kern[dom][0]
    d_gbs = algo[dom] / (d_ms / 1000) / 1e9
    # the headline roofline: the whole step against the scope's algorithmic bytes, 12 B per
    # input point (xyz read once) + 16 B per output voxel (centroid + count written)
    path_bytes = 12.0 * n + 16.0 * V
    path_gbs = path_bytes / (ms / 1000) / 1e9
    traffic = profiled_traffic({"point": n, "valid_point": nvalid, "voxel": V})

    # end to end: pinned host cloud in, key/centroid/count rows out, through the C ABI
    keys_h = torch.empty(n, dtype=torch.int64).pin_memory()
    cent_h = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    cnt_h = torch.empty(n, dtype=torch.int32).pin_memory()
    nv_h = torch.empty(1, dtype=torch.int64).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    copy_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(e2e_steps)]

    def e2e_step(ev=None):
        if ev:
            ev[0].record(stream)
        xyz.copy_(xyz_host, non_blocking=True)
        if ev:
            ev[1].record(stream)
        call()
        nv_h.copy_(buf.num_voxels, non_blocking=True)
        stream.synchronize()
        v = int(nv_h.item())
        if ev:
            ev[2].record(stream)
        keys_h[:v].copy_(buf.keys[:v], non_blocking=True)
        cent_h[:v].copy_(buf.centroids[:v], non_blocking=True)
        cnt_h[:v].copy_(buf.counts[:v], non_blocking=True)
        if ev:
            ev[3].record(stream)
        stream.synchronize()
        return 8 + v * (8 + 12 + 4)

    with torch.cuda.stream(stream):
        for _ in range(2):  # untimed: first touch of the pinned buffers by the copy engines
            e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            d2h = e2e_step(copy_ev[k])
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in copy_ev]))
    d2h_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in copy_ev]))
    e2e_seq_s = e2e_s

    # the same steps through the overlapped pipeline (serve.CloudPipeline): step k+1's
    # copy in and decimation run while step k's rows are copied back.  The headline copies
    # back the decimated cloud and its counts (the scope's output bytes, 16 B a voxel);
    # the run with the keys too (24 B a voxel) is reported beside it.
    del keys_h, cent_h, cnt_h
    from paper_2102_11084_gb300 import serve

    def pipeline_run(with_keys):
        pipe = serve.CloudPipeline(n, args.leaf, depth=3, method=args.method, device=dev,
                                   record_timeline=True, with_keys=with_keys)
        for _ in pipe.run([xyz_host] * 3):  # untimed: first touch of the slots' buffers
            pass
        torch.cuda.synchronize()
        n_warm_tl = len(pipe.timeline())
        t0 = time.perf_counter()
        d2h_bytes = 0
        for k_, c_, n_ in pipe.run([xyz_host] * e2e_steps):
            d2h_bytes = 8 + c_.shape[0] * ((8 if with_keys else 0) + 12 + 4)
        sec = (time.perf_counter() - t0) / e2e_steps
        overlap = serve.copy_overlap(pipe.timeline()[n_warm_tl:])
        del pipe
        return max_over_ranks(sec, dev), d2h_bytes, overlap

    e2e_s, d2h_pipe, pipe_overlap = pipeline_run(False)
    e2e_k_s, d2h_pipe_k, pipe_overlap_k = pipeline_run(True)
    e2e_seq_s = max_over_ranks(e2e_seq_s, dev)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    extra = {}
    if not args.no_extra:
        # the same cloud at leaf 0.1 m
        ms01 = _time_ms(lambda: vg.downsample_into(xyz, 0.1, buf, origin_from_min=True), 10)
        v01 = int(buf.num_voxels.item())
        extra["fused_map_50M_leaf0.1"] = {
            "ms": ms01, "points_per_s": n / (ms01 / 1e3), "voxels": v01,
            "roofline_frac": (12.0 * n + 16.0 * v01) / (ms01 / 1e3) / 1e9 / peak}
        # the same cloud through the global LSD radix sort and segmented reduction
        msl = _time_ms(lambda: vg.downsample_into(xyz, args.leaf, buf, origin_from_min=True,
                                                  method="sort_lsd"), 10)
        extra["fused_map_50M_sort_lsd"] = {"ms": msl, "points_per_s": n / (msl / 1e3),
                                           "voxels": int(buf.num_voxels.item())}
        del buf
        torch.cuda.empty_cache()
        extra.update(extra_measurements(args, dev, peak))
    from paper_2102_11084_gb300 import synth as _synth
    cpu = (None if args.no_cpu_baseline else
           cpu_baseline(oracle_timer, _synth.rgbd_frame(640, 480, seed=0)))
    # our kernels per step: extent, keys, first-digit scan, partition, second-digit
    # histogram, bucket scan, partition, bucket kernel, 8 radix passes, count + scan + reduce
    # (the kernels of the grouping not chosen return at once)
    launches_per_step = 1 + 1 + 6 + 8 + 3
    out = {
        "metric": "points/s", "value": total_points / (ms / 1000), "unit": "points/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "points": n, "valid_points": nvalid, "voxels": V,
                   "leaf_m": args.leaf, "method": args.method,
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs (600 MB) larger than L2 (129 MB); no flush"},
        "roofline": {"bound": "hbm", "kernel": "whole step (all kernels of one call)",
                     "achieved": path_gbs, "peak": peak, "unit": "GB/s",
                     "frac": path_gbs / peak, "traffic": traffic,
                     "peak_source": f"hbm_gbs of MEASURED_PEAKS.json ({peak_src})",
                     "algorithmic_bytes_per_launch": path_bytes, "ms_per_launch": ms,
                     "definition": "12 B per input point (xyz read once) + 16 B per output "
                                   "voxel (centroid + count written)"},
        "roofline_kernel": {"kernel": dom, "achieved": d_gbs, "peak": peak, "unit": "GB/s",
                            "frac": d_gbs / peak, "algorithmic_bytes_per_launch": algo[dom],
                            "ms_per_launch": d_ms, "launches_per_step": kern[dom][1]},
        "stages_ms": st_ms,
        "sort_passes": passes,
        "layout": "narrow (32-bit keys, packed offsets)" if narrow else "wide (64-bit keys, index)",
        "grouping": ("partition passes over the top key bits, every bucket of the low bits "
                     "reduced in one block's shared memory") if bucketed else
                    "every key digit in global radix passes, segmented reduction",
        "cpu_baseline": cpu,
        "e2e": {"value": total_points / e2e_s, "unit": "points/s", "h2d_bytes_per_step": 12 * n,
                "d2h_bytes_per_step": d2h_pipe, "ms_per_step": e2e_s * 1e3,
                "api": ("serve.CloudPipeline (depth 3: copies of neighbouring steps "
                        "overlapped); rows out = centroids + counts, keys stay on the device"),
                "steps": e2e_steps, "warmup": 3,
                "copy_overlap": pipe_overlap,
                "with_keys": {"value": total_points / e2e_k_s, "ms_per_step": e2e_k_s * 1e3,
                              "d2h_bytes_per_step": d2h_pipe_k,
                              "copy_overlap": pipe_overlap_k},
                "sequential": {"value": total_points / e2e_seq_s, "ms_per_step": e2e_seq_s * 1e3,
                               "api": "vg.downsample_into + torch copies, one step at a time",
                               "h2d_ms": h2d_ms, "d2h_ms": d2h_ms,
                               "h2d_GBps": 12 * n / h2d_ms / 1e6,
                               "d2h_GBps": d2h / d2h_ms / 1e6}},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
        "extra": extra,
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_vg(args, rank, world, local)


if __name__ == "__main__":
    main()
