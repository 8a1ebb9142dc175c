"""Host-side logic of the serving loop (no GPU): memory admission and latency stats."""
import collections
from concurrent.futures import Future

import numpy as np

from paper_2102_11084_gb300 import serve, synth


def req(n, t=0.0):
    return serve._Request(0, np.zeros((n, 3), np.float32), 0.05, t, Future())


def test_admission_respects_point_budget_and_frame_limit():
    q = collections.deque([req(100), req(200), req(300), req(50)])
    b = serve.admit(q, max_points=600, max_frames=8)
    assert [r.xyz.shape[0] for r in b] == [100, 200, 300]
    assert [r.xyz.shape[0] for r in q] == [50]        # FIFO: the next batch takes it
    q = collections.deque([req(10) for _ in range(20)])
    assert len(serve.admit(q, max_points=10_000, max_frames=16)) == 16 and len(q) == 4


def test_admission_is_fifo_and_never_overtakes():
    q = collections.deque([req(500), req(700), req(10)])
    b = serve.admit(q, max_points=1000, max_frames=8)
    assert [r.xyz.shape[0] for r in b] == [500]
    assert [r.xyz.shape[0] for r in q] == [700, 10]


def test_empty_queue():
    assert serve.admit(collections.deque(), 100, 4) == []


def test_trace_shape():
    tr = synth.serving_trace(16, 30.0, 10.0, 64, seed=5)
    assert 4000 < len(tr) < 5600                     # 16 x 30 Hz x 10 s, Poisson
    assert all(0 <= r.frame < 64 for r in tr)
    assert all(a.arrival_s <= b.arrival_s for a, b in zip(tr, tr[1:]))
