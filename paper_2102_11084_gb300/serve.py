"""Continuous-batching request loop for voxel-grid decimation of many sensor streams.

Requests (one cloud each, from any number of sensor streams) are queued on the host.
A scheduler thread owns `n_slots` device slots; each slot has its own CUDA stream,
persistent device buffers (input cloud, frame table, outputs, workspace) and pinned host
staging, all allocated once.  Whenever a slot is free the scheduler admits the oldest
waiting requests into it -- as many as fit the slot's point budget and frame limit
(memory admission) -- copies them host-to-device, launches one batched call
(vg_downsample_frames) on the slot's stream and moves on; requests that arrive while
other batches are on the GPU join the next free slot, so one batch's copies overlap
another's decimation (the decimations themselves run one after another).
A completion pass copies each finished batch's rows back and resolves every request's
future with its own voxels and its latency (arrival -> result on the host).

With ``record_timeline=True`` every batch records CUDA events around its copy in, its
decimation and its copy out; ``Server.timeline()`` turns them into intervals on one
device clock and ``copy_overlap()`` measures how much copy time ran under another
batch's decimation.

Every frame of a batch is decimated exactly as it would be alone (same keys, counts
and centroid bits), so a result does not depend on what it was batched with.
"""
from __future__ import annotations

import collections
import ctypes
import threading
import time
from concurrent.futures import Future
from typing import NamedTuple, Optional

import numpy as np
import torch

from . import vg


class Result(NamedTuple):
    keys: np.ndarray        # uint64 [V]
    centroids: np.ndarray   # float32 [V, 3]
    counts: np.ndarray      # uint32 [V]
    origin: np.ndarray      # float32 [3]
    latency_s: float
    batch_frames: int       # how many requests shared the launch


class _Request(NamedTuple):
    stream_id: int
    xyz: np.ndarray
    leaf: float
    arrival: float
    future: Future


class _Slot:
    def __init__(self, device, max_points: int, max_frames: int, method: str):
        self.stream = torch.cuda.Stream(device=device)
        self.max_points = max_points
        self.max_frames = max_frames
        self.flags = vg.method_flag(method) | vg.ORIGIN_FROM_MIN
        cap = max(max_points, 1)
        d = device
        self.xyz = torch.empty((cap, 3), dtype=torch.float32, device=d)
        self.offsets = torch.zeros(max_frames + 1, dtype=torch.int64, device=d)
        self.leaves = torch.ones(max_frames, dtype=torch.float32, device=d)
        self.origins = torch.zeros((max_frames, 3), dtype=torch.float32, device=d)
        self.keys = torch.empty(cap, dtype=torch.int64, device=d)
        self.centroids = torch.empty((cap, 3), dtype=torch.float32, device=d)
        self.counts = torch.empty(cap, dtype=torch.int32, device=d)
        self.out_offsets = torch.zeros(max_frames + 1, dtype=torch.int64, device=d)
        self.error = torch.zeros(1, dtype=torch.int32, device=d)
        nbytes = int(vg.lib().vg_batch_workspace_bytes(cap, max_frames, self.flags))
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=d)
        self.h_xyz = torch.empty((cap, 3), dtype=torch.float32).pin_memory()
        self.h_off_in = torch.zeros(max_frames + 1, dtype=torch.int64).pin_memory()
        self.h_leaf_in = torch.ones(max_frames, dtype=torch.float32).pin_memory()
        self.h_offsets = torch.zeros(max_frames + 1, dtype=torch.int64).pin_memory()
        self.h_origins = torch.zeros((max_frames, 3), dtype=torch.float32).pin_memory()
        self.h_keys = torch.empty(cap, dtype=torch.int64).pin_memory()
        self.h_centroids = torch.empty((cap, 3), dtype=torch.float32).pin_memory()
        self.h_counts = torch.empty(cap, dtype=torch.int32).pin_memory()
        self.h_error = torch.zeros(1, dtype=torch.int32).pin_memory()
        self.done = torch.cuda.Event()
        self.decimated = torch.cuda.Event()
        self.copied = torch.cuda.Event()
        self.batch: list = []
        self.busy = False
        self.copying = False

    def device_bytes(self) -> int:
        ts = [self.xyz, self.offsets, self.leaves, self.origins, self.keys, self.centroids,
              self.counts, self.out_offsets, self.error, self.workspace]
        return sum(t.numel() * t.element_size() for t in ts)

    def launch(self, batch: list, after: Optional[torch.cuda.Event] = None,
               timeline: Optional[list] = None):
        """H2D of the admitted clouds, one batched decimation (behind the event `after`,
        the previous decimation of any slot), D2H of the small tables.  `timeline`: a list
        that receives this batch's timing events."""
        self.batch = batch
        self.busy = True
        ev = None
        if timeline is not None:
            ev = {k: torch.cuda.Event(enable_timing=True)
                  for k in ("h2d0", "h2d1", "dec0", "dec1", "d2h0", "d2h1")}
            timeline.append({"frames": len(batch), "ev": ev, "done": False})
            self.tl_entry = timeline[-1]
        self.ev = ev
        sizes = [r.xyz.shape[0] for r in batch]
        offs = np.zeros(len(batch) + 1, np.int64)
        np.cumsum(sizes, out=offs[1:])
        n = int(offs[-1])
        hx = self.h_xyz.numpy()
        for r, a in zip(batch, offs[:-1]):
            hx[a:a + r.xyz.shape[0]] = r.xyz
        F = len(batch)
        self.h_off_in.numpy()[:F + 1] = offs
        self.h_leaf_in.numpy()[:F] = [r.leaf for r in batch]
        with torch.cuda.stream(self.stream):
            if ev:
                ev["h2d0"].record(self.stream)
            self.xyz[:n].copy_(self.h_xyz[:n], non_blocking=True)
            self.offsets[:F + 1].copy_(self.h_off_in[:F + 1], non_blocking=True)
            self.leaves[:F].copy_(self.h_leaf_in[:F], non_blocking=True)
            if ev:
                ev["h2d1"].record(self.stream)
            if after is not None:
                self.stream.wait_event(after)
            if ev:
                ev["dec0"].record(self.stream)
            st = vg.lib().vg_downsample_frames(
                vg._ptr(self.xyz), n, vg._ptr(self.offsets), F, vg._ptr(self.origins),
                vg._ptr(self.leaves), vg._ptr(self.keys), vg._ptr(self.centroids),
                vg._ptr(self.counts), self.keys.shape[0], vg._ptr(self.out_offsets), None,
                vg._ptr(self.error), vg._ptr(self.workspace), self.workspace.numel(), self.flags,
                ctypes.c_void_p(self.stream.cuda_stream))
            if st != 0:
                raise vg.VGError(st, "vg_downsample_frames")
            self.decimated.record(self.stream)
            if ev:
                ev["dec1"].record(self.stream)
            self.h_offsets[:F + 1].copy_(self.out_offsets[:F + 1], non_blocking=True)
            self.h_origins[:F].copy_(self.origins[:F], non_blocking=True)
            self.h_error.copy_(self.error, non_blocking=True)
            self.done.record(self.stream)
        self.n_frames = F

    def copy_back(self):
        """Issues the copy of the rows back (after `done` fired) and returns at once;
        `copied` fires when they are on the host."""
        F = self.n_frames
        self.err = int(self.h_error[0])
        self.offs = self.h_offsets[:F + 1].numpy().copy()
        v = int(self.offs[-1])
        ev = self.ev
        with torch.cuda.stream(self.stream):
            if ev:
                ev["d2h0"].record(self.stream)
            self.h_keys[:v].copy_(self.keys[:v], non_blocking=True)
            self.h_centroids[:v].copy_(self.centroids[:v], non_blocking=True)
            self.h_counts[:v].copy_(self.counts[:v], non_blocking=True)
            if ev:
                ev["d2h1"].record(self.stream)
            self.copied.record(self.stream)
        self.copying = True

    def finish(self):
        """Splits the copied rows per request and resolves the futures (after `copied`)."""
        self.copied.synchronize()
        if self.ev:
            self.tl_entry["done"] = True
        F = self.n_frames
        err = self.err
        offs = self.offs
        v = int(offs[-1])
        keys = self.h_keys.numpy()[:v].view(np.uint64)
        cents = self.h_centroids.numpy()[:v]
        counts = self.h_counts.numpy()[:v].view(np.uint32)
        origins = self.h_origins.numpy()[:F]
        now = time.perf_counter()
        for f, r in enumerate(self.batch):
            if err:
                r.future.set_exception(vg.VGError(err, "served batch"))
                continue
            a, b = int(offs[f]), int(offs[f + 1])
            r.future.set_result(Result(keys[a:b].copy(), cents[a:b].copy(), counts[a:b].copy(),
                                       origins[f].copy(), now - r.arrival, F))
        self.batch = []
        self.busy = False
        self.copying = False


def admit(queue: collections.deque, max_points: int, max_frames: int) -> list:
    """Memory admission: pops the oldest requests while the batch stays within the slot's
    point budget and frame limit (FIFO: a request that does not fit waits for the next
    slot rather than being overtaken)."""
    batch, pts = [], 0
    while queue and len(batch) < max_frames:
        n = queue[0].xyz.shape[0]
        if pts + n > max_points:
            break
        batch.append(queue.popleft())
        pts += n
    return batch


class Server:
    """Continuous-batching decimation server on one GPU.

    max_points   point budget of one batch (per slot); a request larger than it is refused.
    max_frames   most requests in one batch.
    n_slots      device slots (>= 2 lets a batch's copies overlap another's decimation; with
                 3, one batch can be copied in and another copied out while a third runs).
    mem_budget   device bytes the slots may hold; fewer slots are made if needed.
    """

    def __init__(self, *, max_points: int = 8 * 307_200, max_frames: int = 16, n_slots: int = 3,
                 method: str = "auto", device="cuda", mem_budget: Optional[int] = None,
                 record_timeline: bool = False):
        dev = torch.device(device)
        self._timeline: Optional[list] = [] if record_timeline else None
        self._t0 = None
        if record_timeline:  # the common origin of every batch's event times
            self._t0 = torch.cuda.Event(enable_timing=True)
            self._t0.record(torch.cuda.current_stream(dev))
            self._t0.synchronize()
        self.slots = []
        used = 0
        for _ in range(max(1, n_slots)):
            s = _Slot(dev, max_points, max_frames, method)
            if mem_budget is not None and self.slots and used + s.device_bytes() > mem_budget:
                del s
                break
            used += s.device_bytes()
            self.slots.append(s)
        self.device_bytes = used
        self.max_points = max_points
        self.max_frames = max_frames
        self._q = collections.deque()
        self._last_decimated: Optional[torch.cuda.Event] = None
        self._cv = threading.Condition()
        self._stop = False
        self.batches = 0
        self.points = 0
        self._thread = threading.Thread(target=self._loop, name="vg-serve", daemon=True)
        self._thread.start()

    def submit(self, stream_id: int, xyz: np.ndarray, leaf: float,
               arrival: Optional[float] = None) -> Future:
        xyz = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
        fut: Future = Future()
        if xyz.shape[0] > self.max_points:
            fut.set_exception(ValueError("cloud larger than a batch's point budget"))
            return fut
        req = _Request(stream_id, xyz, float(leaf), time.perf_counter() if arrival is None else arrival,
                       fut)
        with self._cv:
            self._q.append(req)
            self._cv.notify()
        return fut

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify()
        self._thread.join()

    def timeline(self) -> list:
        """Per finished batch (record_timeline=True): ms from the server's start on the
        device clock of its copy in, decimation and copy out, as (start, end) pairs."""
        if self._timeline is None:
            raise ValueError("the server was made without record_timeline")
        return _intervals(self._timeline, self._t0)

    def _admit(self) -> list:
        return admit(self._q, self.max_points, self.max_frames)

    def _loop(self):
        torch.cuda.set_device(self.slots[0].xyz.device)
        while True:
            progressed = False
            for s in self.slots:
                if s.busy and not s.copying and s.done.query():
                    s.copy_back()  # the rows travel back while other batches run
                    progressed = True
                if s.copying and s.copied.query():
                    s.finish()
                    progressed = True
            with self._cv:
                if self._stop and not self._q and not any(s.busy for s in self.slots):
                    return
                free = [s for s in self.slots if not s.busy]
                batch = self._admit() if (free and self._q) else []
                if not batch and not progressed and not any(s.busy for s in self.slots):
                    self._cv.wait(timeout=0.05)
                    continue
            if batch:
                try:
                    # batches copy in and out concurrently, but decimate one at a time: two
                    # GPU-filling persistent grids of chained-scan kernels at once make each
                    # other's blocks wait on tiles that cannot get an SM
                    free[0].launch(batch, self._last_decimated, self._timeline)
                    self._last_decimated = free[0].decimated
                    self.batches += 1
                    self.points += sum(r.xyz.shape[0] for r in batch)
                except Exception as e:  # fail this batch's requests, keep serving
                    for r in batch:
                        if not r.future.done():
                            r.future.set_exception(e)
                    free[0].busy = False
            elif not progressed:
                time.sleep(0.0002)


def replay(server: Server, trace, pool, leaf: float, *, realtime: bool = True):
    """Feeds a request trace (synth.serving_trace) into the server; returns the results."""
    t0 = time.perf_counter()
    futs = []
    for r in trace:
        if realtime:
            delay = t0 + r.arrival_s - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
        futs.append((r, server.submit(r.stream, pool[r.frame], leaf)))
    out = [(r, f.result()) for r, f in futs]
    return out, time.perf_counter() - t0


def _intervals(timeline: list, t0) -> list:
    out = []
    for b in list(timeline):
        if not b["done"]:
            continue  # not finished (or failed before its events were recorded)
        t = {k: t0.elapsed_time(e) for k, e in b["ev"].items()}
        out.append({"frames": b["frames"], "h2d": (t["h2d0"], t["h2d1"]),
                    "decimate": (t["dec0"], t["dec1"]), "d2h": (t["d2h0"], t["d2h1"])})
    return out


def _union_overlap(a: tuple, spans: list) -> float:
    """Length of interval a covered by the union of spans."""
    lo, hi = a
    cut = sorted((max(lo, s), min(hi, e)) for s, e in spans if min(hi, e) > max(lo, s))
    total, end = 0.0, lo
    for s, e in cut:
        s = max(s, end)
        if e > s:
            total += e - s
            end = e
    return total


def copy_overlap(timeline: list) -> dict:
    """How much of the batches' copy time (in and out) ran while another batch was being
    decimated: overlapped ms / copy ms, from Server.timeline().  The decimation time is
    reported beside it: at most that much copy time of the other batches can be hidden
    per copy direction, so where copies take longer than decimations the fraction is
    bounded by their ratio."""
    copy_ms = over_ms = 0.0
    dec_ms = sum(max(0.0, b["decimate"][1] - b["decimate"][0]) for b in timeline)
    for i, b in enumerate(timeline):
        others = [o["decimate"] for j, o in enumerate(timeline) if j != i]
        for key in ("h2d", "d2h"):
            s, e = b[key]
            copy_ms += max(0.0, e - s)
            over_ms += _union_overlap((s, e), others)
    return {"batches": len(timeline), "copy_ms": copy_ms, "overlapped_ms": over_ms,
            "decimate_ms": dec_ms, "fraction": over_ms / copy_ms if copy_ms > 0 else 0.0}


def latency_stats(results) -> dict:
    lat = np.array([res.latency_s for _, res in results]) * 1000.0
    pts = sum(int(res.counts.sum()) for _, res in results)
    return {"requests": len(results), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
            "valid_points": pts,
            "mean_batch_frames": float(np.mean([res.batch_frames for _, res in results]))}


class CloudPipeline:
    """Decimates a sequence of large host clouds with the copies overlapped.

    ``depth`` device slots, each with its own stream, input buffer, outputs, workspace
    and pinned host rows.  Cloud k goes to slot k % depth: host-to-device copy, one
    vg_downsample, then -- once the host has read its voxel count -- the copy of its V
    rows back, all on the slot's stream.  While cloud k's rows travel back, later clouds
    are copied in and decimated on the other slots, so a sequence runs at the pace of
    its slowest stage instead of the sum of the three.

    ``run(clouds)`` yields, in order, (keys uint64 [V], centroids float32 [V, 3],
    counts uint32 [V]) numpy views of pinned host memory; a view stays valid until the
    pipeline takes ``depth`` more clouds.  Every cloud's result is the plain call's,
    bit for bit.  With ``with_keys=False`` the keys stay on the device (keys is None):
    the decimated cloud and its point counts, 16 bytes a voxel instead of 24, come back.

    The copies of different clouds overlap, their decimations do not: a cloud's
    decimation starts only after the previous cloud's has finished.  Two decimations at
    once would put two persistent, GPU-filling grids of chained-scan kernels on the
    device together, whose blocks then wait on tiles the other grid keeps off the SMs
    (measured: 18 ms a step instead of 5.7 when the timing let them meet).
    """

    def __init__(self, max_points: int, leaf: float, *, depth: int = 3, method: str = "auto",
                 device="cuda", record_timeline: bool = False, with_keys: bool = True):
        self.leaf = float(leaf)
        self.with_keys = bool(with_keys)
        self._timeline: Optional[list] = [] if record_timeline else None
        self._t0 = None
        if record_timeline:  # the common origin of every cloud's event times
            self._t0 = torch.cuda.Event(enable_timing=True)
            self._t0.record(torch.cuda.current_stream(torch.device(device)))
            self._t0.synchronize()
        self.method = method
        self.max_points = int(max_points)
        dev = torch.device(device)
        self.device = dev
        flags = vg.method_flag(method)
        self._last_decimated = None  # event after the latest issued decimation
        self.slots = []
        for _ in range(max(2, int(depth))):
            s = {"stream": torch.cuda.Stream(device=dev),
                 "decimated": torch.cuda.Event(),
                 "xyz": torch.empty((self.max_points, 3), dtype=torch.float32, device=dev),
                 "buf": vg.alloc_buffers(self.max_points, dev, flags=flags),
                 "keys": (torch.empty(self.max_points, dtype=torch.int64).pin_memory()
                          if self.with_keys else None),
                 "cents": torch.empty((self.max_points, 3), dtype=torch.float32).pin_memory(),
                 "counts": torch.empty(self.max_points, dtype=torch.int32).pin_memory(),
                 "nv": torch.zeros(1, dtype=torch.int64).pin_memory(),
                 "err": torch.zeros(1, dtype=torch.int32).pin_memory(),
                 "counted": torch.cuda.Event(), "done": torch.cuda.Event(), "v": 0,
                 "state": "free", "ev": None}
            self.slots.append(s)

    def _launch(self, s, host: torch.Tensor):
        n = host.shape[0]
        if n > self.max_points:
            raise ValueError("cloud larger than the pipeline's max_points")
        ev = None
        if self._timeline is not None:
            ev = {k: torch.cuda.Event(enable_timing=True)
                  for k in ("h2d0", "h2d1", "dec0", "dec1", "d2h0", "d2h1")}
            self._timeline.append({"frames": 1, "ev": ev, "done": False})
            s["tl"] = self._timeline[-1]
        s["ev"] = ev
        with torch.cuda.stream(s["stream"]):
            if ev:
                ev["h2d0"].record(s["stream"])
            s["xyz"][:n].copy_(host, non_blocking=True)
            if ev:
                ev["h2d1"].record(s["stream"])
            if self._last_decimated is not None:  # one decimation on the device at a time
                s["stream"].wait_event(self._last_decimated)
            if ev:
                ev["dec0"].record(s["stream"])
            vg.downsample_into(s["xyz"][:n], self.leaf, s["buf"], origin_from_min=True,
                               method=self.method, stream=s["stream"])
            s["decimated"].record(s["stream"])
            if ev:
                ev["dec1"].record(s["stream"])
            self._last_decimated = s["decimated"]
            s["nv"].copy_(s["buf"].num_voxels, non_blocking=True)
            s["err"].copy_(s["buf"].error, non_blocking=True)
            s["counted"].record(s["stream"])
        s["state"] = "counting"

    def _copy_back(self, s):
        s["counted"].synchronize()
        if int(s["err"][0]):
            raise vg.VGError(int(s["err"][0]), "pipeline cloud")
        v = int(s["nv"][0])
        s["v"] = v
        b = s["buf"]
        ev = s["ev"]
        with torch.cuda.stream(s["stream"]):
            if ev:
                ev["d2h0"].record(s["stream"])
            if self.with_keys:
                s["keys"][:v].copy_(b.keys[:v], non_blocking=True)
            s["cents"][:v].copy_(b.centroids[:v], non_blocking=True)
            s["counts"][:v].copy_(b.counts[:v], non_blocking=True)
            if ev:
                ev["d2h1"].record(s["stream"])
            s["done"].record(s["stream"])
        s["state"] = "copying"

    def _result(self, s):
        s["done"].synchronize()
        if s["ev"]:
            s["tl"]["done"] = True
        v = s["v"]
        s["state"] = "free"
        keys = s["keys"].numpy()[:v].view(np.uint64) if self.with_keys else None
        return keys, s["cents"].numpy()[:v], s["counts"].numpy()[:v].view(np.uint32)

    def timeline(self) -> list:
        """Per cloud handed out (record_timeline=True): ms from the pipeline's start on the
        device clock of its copy in, decimation and copy out, as (start, end) pairs."""
        if self._timeline is None:
            raise ValueError("the pipeline was made without record_timeline")
        return _intervals(self._timeline, self._t0)

    def run(self, clouds):
        """clouds: iterable of float32 [N, 3] CPU tensors (pinned for overlap)."""
        # Every free slot takes the next cloud at once (its copy in queued behind the
        # others'), and a cloud's rows start back as soon as its voxel count is in; the
        # host waits only when the next cloud needs a slot whose cloud is not handed out.
        order = collections.deque()
        k = 0
        for host in clouds:
            s = self.slots[k % len(self.slots)]
            while s["state"] != "free":  # the slot's previous cloud is handed out first
                o = order.popleft()
                if o["state"] == "counting":
                    self._copy_back(o)
                yield self._result(o)
            self._launch(s, host)
            order.append(s)
            k += 1
            for o in order:  # copies back of the clouds counted so far, oldest first
                if o["state"] == "counting":
                    if not o["counted"].query():
                        break
                    self._copy_back(o)
        while order:
            o = order.popleft()
            if o["state"] == "counting":
                self._copy_back(o)
            yield self._result(o)
