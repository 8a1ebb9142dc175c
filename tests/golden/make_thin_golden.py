"""Writes thin_640x480.txt: the oracle's result of the neighbour-count thinning loop
(reading R16 of arXiv 2102.11084 Sec. II-C, Algorithm 1 with Eq. 1) on the 640x480
RGB-D frame of seed 0, cell = radius 0.05 m, threshold 20, batches of 1000 points,
priority = the seed-5 permutation.  Only the oracle runs here (about three minutes on
one core); the GPU test compares vg_thin's keep flags with the stored digest.

    python tests/golden/make_thin_golden.py
"""
import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2102_11084_gb300 import synth  # noqa: E402

CELL, THRESHOLD, BATCH = 0.05, 20, 1000


def inputs():
    x = synth.rgbd_frame(640, 480, seed=0)
    pr = np.random.Generator(np.random.PCG64(5)).permutation(x.shape[0]).astype(np.uint32)
    return x, pr


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def main():
    x, pr = inputs()
    keep, passes, st = oracle.thin(x, CELL, THRESHOLD, pr, batch=BATCH)
    assert st == 0
    with open(os.path.join(HERE, "thin_640x480.txt"), "w") as f:
        f.write("# Oracle result of the neighbour-count thinning loop (reading R16; arXiv\n"
                "# 2102.11084 Sec. II-C, Algorithm 1, Eq. 1) on the 640x480 RGB-D frame of seed 0,\n"
                f"# cell = radius {CELL} m, threshold {THRESHOLD}, batch {BATCH}, priority = the\n"
                "# seed-5 permutation.  Written by make_thin_golden.py (oracle only).  Digests are\n"
                "# SHA-256 of the float32 cloud, the uint32 priorities and np.packbits(keep).\n")
        f.write(f"cloud_sha256 {digest(x)}\n")
        f.write(f"priority_sha256 {digest(pr)}\n")
        f.write(f"passes {passes}\n")
        f.write(f"kept {int(keep.sum())}\n")
        f.write(f"keep_sha256 {digest(np.packbits(keep))}\n")


if __name__ == "__main__":
    main()
