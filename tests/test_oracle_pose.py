"""Pins of the oracle's posed-cloud reading R12 (Sec. II-C: the camera cloud is taken
into the global frame, and the height is limited there, before the voxel filter).

Special cases with exact arithmetic pin the layout of [R|t] (row-major), the sign and
place of t, that the limit applies to z' after the pose and is inclusive; the general
case is the definition evaluated step by step in numpy binary32."""
import numpy as np
import pytest

import oracle
from paper_2102_11084_gb300 import synth


def cloud(n=3000, seed=5):
    return synth.random_cloud(n, seed=seed, extent=4.0, nan_frac=0.05, inf_frac=0.01)


def same(a, b):
    """Equal as binary32 values, NaN rows matching NaN rows."""
    return np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(
        np.nan_to_num(a, nan=0.0), np.nan_to_num(b, nan=0.0))


def rows_valid(a):
    return np.isfinite(a).all(axis=1)


def test_identity_keeps_every_point():
    x = cloud()
    out = oracle.pose(x, np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32))
    ok = rows_valid(x)
    assert same(out[ok], x[ok]) and np.isnan(out[~ok]).all()
    assert same(oracle.pose(x), np.where(ok[:, None], x, np.nan))


def test_quarter_turn_about_z_plus_translation_is_exact():
    # R = [[0,-1,0],[1,0,0],[0,0,1]]: every product is exact and the sums collapse to one
    # rounding each, so x' = fl(-y + tx), y' = fl(x + ty), z' = fl(z + tz).
    x = cloud(seed=6)
    t = np.float32([0.25, -1.5, 3.0])
    rt = np.array([[0, -1, 0, t[0]], [1, 0, 0, t[1]], [0, 0, 1, t[2]]], np.float32)
    out = oracle.pose(x, rt)
    ok = rows_valid(x)
    want = np.stack([-x[:, 1] + t[0], x[:, 0] + t[1], x[:, 2] + t[2]], axis=1).astype(np.float32)
    assert same(out[ok], want[ok]) and np.isnan(out[~ok]).all()


def test_height_limit_is_inclusive_and_after_the_pose():
    # quarter turn about x: z' = y + 0.5; the band is checked on z', ends included
    x = cloud(seed=7)
    lo, hi = np.float32(-1.0), np.float32(1.25)
    x[0] = [0.1, lo - 0.5, 0.3]                       # z' == lo exactly: kept
    x[1] = [0.2, hi - 0.5, 0.3]                       # z' == hi exactly: kept
    x[2] = [0.3, np.nextafter(lo, np.float32(-9)) - np.float32(0.5), 0.3]  # z' one ulp below
    x[3] = [0.4, np.nextafter(hi, np.float32(9)) - np.float32(0.5), 0.3]   # z' one ulp above
    rt = np.array([[1, 0, 0, 0], [0, 0, -1, 0], [0, 1, 0, 0.5]], np.float32)
    out = oracle.pose(x, rt, [lo, hi])
    zp = (x[:, 1] + np.float32(0.5)).astype(np.float32)
    keep = rows_valid(x) & (zp >= lo) & (zp <= hi)
    assert keep[0] and keep[1] and not keep[2] and not keep[3]
    assert np.array_equal(rows_valid(out), keep)
    assert same(out[keep], np.stack([x[:, 0], -x[:, 2], zp], axis=1)[keep])


def test_general_pose_matches_stepwise_binary32():
    x = cloud(seed=8)
    rng = np.random.Generator(np.random.PCG64(9))
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, a, b, c = q
    R = np.array([[1 - 2 * (b * b + c * c), 2 * (a * b - c * w), 2 * (a * c + b * w)],
                  [2 * (a * b + c * w), 1 - 2 * (a * a + c * c), 2 * (b * c - a * w)],
                  [2 * (a * c - b * w), 2 * (b * c + a * w), 1 - 2 * (a * a + b * b)]])
    rt = np.concatenate([R, rng.uniform(-3, 3, size=(3, 1))], axis=1).astype(np.float32)
    out = oracle.pose(x, rt, [-2.0, 2.0])
    f = np.float32
    g = np.empty_like(x)
    for ax in range(3):
        r = rt[ax]
        acc = (r[0] * x[:, 0]).astype(f)
        acc = (acc + (r[1] * x[:, 1]).astype(f)).astype(f)
        acc = (acc + (r[2] * x[:, 2]).astype(f)).astype(f)
        g[:, ax] = (acc + r[3]).astype(f)
    keep = rows_valid(g) & (g[:, 2] >= f(-2.0)) & (g[:, 2] <= f(2.0))
    assert 0 < keep.sum() < rows_valid(x).sum()
    assert np.array_equal(rows_valid(out), keep) and same(out[keep], g[keep])


def test_posed_decimation_is_the_plain_one_on_the_posed_cloud():
    x = cloud(seed=10)
    rt = np.array([[0, -1, 0, 2.0], [1, 0, 0, 1.0], [0, 0, 1, 0.0]], np.float32)
    a = oracle.downsample_posed(x, 0.2, rt, [-1.0, 1.5])
    b = oracle.downsample(oracle.pose(x, rt, [-1.0, 1.5]), 0.2)
    assert np.array_equal(a.keys, b.keys) and np.array_equal(a.counts, b.counts)
    assert np.array_equal(a.centroids, b.centroids)
    assert int(a.counts.sum()) == int(rows_valid(oracle.pose(x, rt, [-1.0, 1.5])).sum())
