"""GPU parity of the neighbour-count thinning loop (vg_thin) against the oracle's reading
R16 of the paper's own filter (Sec. II-C, Algorithm 1; Eq. 1): the keep flag of every
point, the number kept and the number of passes must be identical."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_11084_gb300 import synth, vg

pytestmark = pytest.mark.gpu


def ranks(n, seed):
    return np.random.Generator(np.random.PCG64(seed)).permutation(n).astype(np.uint32)


def run(x, cell, t, pr, **kw):
    return vg.thin(torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda(), cell, t,
                   torch.from_numpy(pr.view(np.int32)).cuda(), **kw)


@pytest.mark.parametrize("t,batch,radius", [(20, 200, None), (8, 400, None), (12, 300, 0.03),
                                            (40, 1000, None)])
def test_rgbd_frame_matches_oracle(t, batch, radius):
    x = synth.rgbd_frame(160, 120, seed=11)
    pr = ranks(x.shape[0], seed=t)
    keep, passes, st = oracle.thin(x, 0.05, t, pr, radius=radius, batch=batch)
    assert st == 0 and 0 < keep.sum() < np.isfinite(x).all(axis=1).sum()
    res = run(x, 0.05, t, pr, radius=radius, batch=batch)
    assert np.array_equal(res.keep.cpu().numpy(), keep)
    assert res.num_kept == int(keep.sum()) and res.passes == passes


@pytest.mark.parametrize("m,t,k", [(25, 4, 3), (10, 3, 1000), (40, 0, 7)])
def test_clique(m, t, k):
    rng = np.random.Generator(np.random.PCG64(m))
    x = (np.float32([1.03, 2.07, 0.51]) + rng.uniform(-0.004, 0.004, (m, 3))).astype(np.float32)
    pr = ranks(m, seed=t)
    keep, passes, _ = oracle.thin(x, 0.05, t, pr, batch=k)
    res = run(x, 0.05, t, pr, batch=k)
    assert np.array_equal(res.keep.cpu().numpy(), keep) and res.passes == passes


def test_ragged_invalid_and_untouched_clouds():
    for n in (1, 2, 1000, 4097):
        x = synth.random_cloud(n, seed=n, extent=0.4, nan_frac=0.1, inf_frac=0.02)
        pr = ranks(n, seed=n)
        keep, passes, _ = oracle.thin(x, 0.05, 6, pr, batch=37)
        res = run(x, 0.05, 6, pr, batch=37)
        assert np.array_equal(res.keep.cpu().numpy(), keep) and res.passes == passes
    y = synth.random_cloud(3000, seed=9, extent=0.3, nan_frac=0.1)
    res = run(y, 0.05, 10 ** 6, ranks(3000, 1), batch=10)
    assert np.array_equal(res.keep.cpu().numpy(), np.isfinite(y).all(axis=1))
    assert res.passes == 1
    empty = run(np.zeros((0, 3), np.float32), 0.05, 1, np.zeros(0, np.uint32))
    assert empty.num_kept == 0


def test_rgbd_640x480_bench_parameters():
    """The bench's configuration (640x480 frame, cell 0.05 m, threshold 20, batches of
    1000): keep flags, kept count and passes against the oracle's result stored in
    tests/golden/thin_640x480.txt (written by make_thin_golden.py from the oracle alone);
    if this machine generates a different cloud, the oracle runs here instead."""
    import hashlib
    import os
    import sys
    golden = os.path.join(os.path.dirname(__file__), "golden")
    sys.path.insert(0, golden)
    import make_thin_golden as mk
    rec = {}
    with open(os.path.join(golden, "thin_640x480.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                rec[k] = v
    x, pr = mk.inputs()
    res = run(x, mk.CELL, mk.THRESHOLD, pr, batch=mk.BATCH)
    keep = res.keep.cpu().numpy().astype(bool)
    if mk.digest(x) == rec["cloud_sha256"] and mk.digest(pr) == rec["priority_sha256"]:
        assert res.passes == int(rec["passes"]) and res.num_kept == int(rec["kept"])
        assert mk.digest(np.packbits(keep)) == rec["keep_sha256"]
    else:  # (the stored result belongs to another cloud)
        ref, passes, st = oracle.thin(x, mk.CELL, mk.THRESHOLD, pr, batch=mk.BATCH)
        assert st == 0 and res.passes == passes and np.array_equal(keep, ref)
