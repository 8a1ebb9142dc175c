"""Pins of the CPU oracle against facts other than itself (no GPU needed).

Each test pins one part of the oracle (arXiv 2102.11084 Sec. II-C: cell key, cell
table sorted by cell, one output point per occupied cell) with an independent check:
hand-worked golden values, O(N^2) brute-force grouping done in numpy binary32,
closed forms, special cases and invariants.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2102_11084_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _decode_morton(key: int):
    """Inverse of the key layout (bit 3b -> x bit b, 3b+1 -> y, 3b+2 -> z)."""
    ijk = [0, 0, 0]
    for bit in range(63):
        if (key >> bit) & 1:
            ijk[bit % 3] |= 1 << (bit // 3)
    return tuple(ijk)


def _numpy_ijk(xyz, origin, leaf):
    """binary32 voxel indices computed by numpy (IEEE single ops, independent code)."""
    p = np.asarray(xyz, np.float32)
    o = np.asarray(origin, np.float32)
    t = np.subtract(p, o, dtype=np.float32)
    q = np.divide(t, np.float32(leaf), dtype=np.float32)
    return np.floor(q).astype(np.int64)


def _valid_rows(xyz):
    return np.isfinite(np.asarray(xyz)).all(axis=1)


def test_morton_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "morton_keys.txt"))
            if l.strip() and not l.startswith("#")]
    ijk = np.array([[int(r[0]), int(r[1]), int(r[2])] for r in rows], np.float64)
    want = [int(r[3]) for r in rows]
    # a point at the centre of voxel ijk with origin 0, leaf 1 lands in voxel ijk
    pts = (ijk + 0.5).astype(np.float32)
    keys, got_ijk, valid, st = oracle.keys(pts, np.zeros(3, np.float32), 1.0)
    assert st == 0 and valid.all()
    assert [int(k) for k in keys] == want
    assert (got_ijk == ijk.astype(np.int64)).all()
    for k, (i, j, l) in zip(want, ijk.astype(int)):
        assert _decode_morton(k) == (i, j, l)


def _read_tiny():
    sec = None
    data = {"points": [], "voxels": [], "point_to_voxel": []}
    meta = {}
    for line in open(os.path.join(GOLDEN, "tiny_cloud.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line in data:
            sec = line
            continue
        parts = line.split()
        if sec is None:
            meta[parts[0]] = parts[1:]
        else:
            data[sec].append(parts)
    return meta, data


def test_tiny_hand_worked():
    meta, data = _read_tiny()
    leaf = float(meta["leaf"][0])
    origin = np.array([float(v) for v in meta["origin"]], np.float32)
    pts = np.array([[float(v) for v in r] for r in data["points"]], np.float32)
    d = oracle.downsample(pts, leaf, origin)
    assert d.status == 0
    want = data["voxels"]
    assert [int(k) for k in d.keys] == [int(r[0]) for r in want]
    assert [int(c) for c in d.counts] == [int(r[1]) for r in want]
    for row, c in zip(want, d.centroids):
        for a in range(3):
            assert abs(c[a] - float(Fraction(row[2 + a]))) < 1e-15
    assert d.point_to_voxel.tolist() == [int(v) for v in data["point_to_voxel"][0]]


@pytest.mark.parametrize("seed,leaf,clusters", [(0, 0.05, 0), (1, 0.2, 0), (2, 0.05, 20),
                                                (3, 0.013, 7), (4, 0.5, 0)])
def test_bruteforce_grouping(seed, leaf, clusters):
    xyz = synth.random_cloud(1500, seed, extent=2.0, nan_frac=0.05, inf_frac=0.01,
                             clusters=clusters, cluster_sigma=0.02)
    valid = _valid_rows(xyz)
    origin = xyz[valid].min(axis=0)
    d = oracle.downsample(xyz, leaf, origin)
    assert d.status == 0
    ijk = np.zeros((xyz.shape[0], 3), np.int64)
    ijk[valid] = _numpy_ijk(xyz[valid], origin, leaf)
    idx = np.nonzero(valid)[0]
    # O(N^2): same voxel (numpy binary32) <=> same output row (oracle)
    same_np = (ijk[idx][:, None, :] == ijk[idx][None, :, :]).all(axis=2)
    same_or = d.point_to_voxel[idx][:, None] == d.point_to_voxel[idx][None, :]
    assert (same_np == same_or).all()
    assert (d.point_to_voxel[~valid] == -1).all()
    # counts and centroids per output row from the brute-force membership
    assert int(d.counts.sum()) == len(idx)
    for r in range(len(d.keys)):
        members = idx[d.point_to_voxel[idx] == r]
        assert len(members) == int(d.counts[r])
        for a in range(3):
            exact = math.fsum(float(x) for x in xyz[members, a]) / len(members)
            assert abs(d.centroids[r, a] - exact) <= 1e-12 * max(1.0, abs(exact))
        # the key decodes to the voxel indices numpy computed for the members
        assert _decode_morton(int(d.keys[r])) == tuple(int(v) for v in ijk[members[0]])
    # ascending, unique keys
    assert (np.diff(d.keys.astype(np.float64)) > 0).all() or len(d.keys) < 2
    assert np.all(d.keys[1:] > d.keys[:-1])


def test_face_points_go_up():
    leaf = 0.25  # power of two: o + k*leaf is exact, so (p - o)/leaf is an integer
    o = np.array([1.0, -2.0, 0.5], np.float32)
    pts = np.array([o + np.float32(leaf) * np.float32(k) for k in range(5)], np.float32)
    keys, ijk, valid, st = oracle.keys(pts, o, leaf)
    assert st == 0 and valid.all()
    assert ijk[:, 0].tolist() == [0, 1, 2, 3, 4]
    # just below a face stays in the lower voxel
    below = np.nextafter(pts[1], np.float32(-np.inf)).astype(np.float32)[None]
    _, ijk2, _, _ = oracle.keys(below, o, leaf)
    assert ijk2[0].tolist() == [0, 0, 0]


def test_special_cases():
    o = np.zeros(3, np.float32)
    # empty cloud
    d = oracle.downsample(np.zeros((0, 3), np.float32), 0.1, o)
    assert len(d.keys) == 0 and d.status == 0
    # all invalid (NaN and +-Inf on single axes)
    bad = np.array([[np.nan, 0, 0], [0, np.inf, 0], [0, 0, -np.inf], [np.nan] * 3], np.float32)
    d = oracle.downsample(bad, 0.1, o)
    assert len(d.keys) == 0 and (d.point_to_voxel == -1).all()
    org, nvalid = oracle.origin(bad)
    assert nvalid == 0 and (org == 0).all()
    # single point: its own centroid; origin = the point -> key 0
    p = np.array([[3.25, -1.5, 7.0]], np.float32)
    d = oracle.downsample(p, 0.05)
    assert d.keys.tolist() == [0] and d.counts.tolist() == [1]
    assert (d.centroids[0] == p[0].astype(np.float64)).all()


def test_leaf_much_larger_than_extent():
    xyz = synth.random_cloud(3000, 7, extent=1.0, nan_frac=0.1)
    d = oracle.downsample(xyz, 1000.0)
    valid = xyz[_valid_rows(xyz)]
    assert len(d.keys) == 1 and int(d.counts[0]) == len(valid)
    for a in range(3):
        exact = math.fsum(float(x) for x in valid[:, a]) / len(valid)
        assert abs(d.centroids[0, a] - exact) <= 1e-13


def test_leaf_much_smaller_than_spacing():
    g = np.stack(np.meshgrid(np.arange(6), np.arange(5), np.arange(4), indexing="ij"), -1)
    xyz = (g.reshape(-1, 3) * 0.5 + 0.1).astype(np.float32)
    d = oracle.downsample(xyz, 0.01)
    assert len(d.keys) == xyz.shape[0] and (d.counts == 1).all()
    # each centroid is exactly its point
    got = np.sort(d.centroids.view([("x", "f8"), ("y", "f8"), ("z", "f8")]).ravel())
    want = np.sort(xyz.astype(np.float64).view([("x", "f8"), ("y", "f8"), ("z", "f8")]).ravel())
    assert (got == want).all()


def test_range_error():
    o = np.zeros(3, np.float32)
    far = np.array([[0.0, 0.0, 0.0], [0.1 * 2**21 + 1.0, 0.0, 0.0]], np.float32)
    d = oracle.downsample(far, 0.1, o)
    assert d.status == oracle.STATUS_RANGE
    below = np.array([[-1.0, 0.0, 0.0]], np.float32)
    assert oracle.downsample(below, 0.1, o).status == oracle.STATUS_RANGE
    # the last index inside the range is accepted
    edge = np.array([[2**21 - 1 + 0.5, 0.0, 0.0]], np.float32)
    d = oracle.downsample(edge, 1.0, o)
    assert d.status == 0 and int(d.keys[0]) == 1317624576693539401


def test_capacity():
    xyz = synth.random_cloud(500, 3, extent=1.0, nan_frac=0.0)
    d = oracle.downsample(xyz, 0.05)
    small = oracle.downsample(xyz, 0.05, cap=10)
    assert small.status == oracle.STATUS_CAPACITY
    assert (small.keys == d.keys[:10]).all()


def test_origin_is_min_over_valid_rows():
    xyz = synth.random_cloud(4000, 11, extent=3.0, nan_frac=0.2, inf_frac=0.05,
                             offset=(-1.0, 2.0, -5.0))
    o, nvalid = oracle.origin(xyz)
    valid = xyz[_valid_rows(xyz)]
    assert nvalid == len(valid)
    assert (o == valid.min(axis=0)).all()


@pytest.mark.parametrize("leaf", [0.05, 0.02])
def test_invariants_on_rgbd_frame(leaf):
    xyz = synth.rgbd_frame(160, 120, seed=3)
    d = oracle.downsample(xyz, leaf)
    valid = _valid_rows(xyz)
    assert int(d.counts.sum()) == int(valid.sum())
    # every centroid lies inside its voxel box (slack: a few binary32 ulps)
    ijk = np.array([_decode_morton(int(k)) for k in d.keys], np.float64)
    lo = d.origin.astype(np.float64) + ijk * leaf
    slack = 1e-5
    assert (d.centroids >= lo - slack).all() and (d.centroids <= lo + leaf + slack).all()


def test_idempotence():
    xyz = synth.rgbd_frame(160, 120, seed=4)
    leaf = 0.05
    d = oracle.downsample(xyz, leaf)
    c32 = d.centroids.astype(np.float32)
    again = oracle.downsample(c32, leaf, d.origin)
    # a centroid within one ulp of a face may flip voxel; flag and count those
    ijk = np.array([_decode_morton(int(k)) for k in d.keys], np.float64)
    q = (c32.astype(np.float64) - d.origin.astype(np.float64)) / leaf - ijk
    near_face = ((q < 1e-5) | (q > 1 - 1e-5)).any(axis=1)
    assert near_face.sum() == 0
    assert (again.keys == d.keys).all() and (again.counts == 1).all()
    assert np.abs(again.centroids - d.centroids).max() <= 1e-5


@pytest.mark.parametrize("levels", [4])
def test_pyramid_equals_direct_decimation(levels):
    xyz = synth.rgbd_frame(320, 240, seed=5)
    base = 0.01
    pyr, d0 = oracle.pyramid(xyz, base, levels)
    for k in range(levels):
        leaf_k = float(np.float32(2**k) * np.float32(base))
        direct = oracle.downsample(xyz, leaf_k, d0.origin)
        keys, cents, counts = pyr[k]
        assert (keys == direct.keys).all()
        assert (counts == direct.counts).all()
        assert np.abs(cents - direct.centroids).max() <= 1e-12


def test_pyramid_merge_hand_worked():
    # children keys 0..7 share parent 0; key 8 -> parent 1; counts weight the mean
    keys = np.array([0, 5, 8], np.uint64)
    cents = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 3.0], [4.0, 4.0, 4.0]])
    counts = np.array([1, 3, 2], np.uint64)
    k, c, n = oracle.pyramid_merge(keys, cents, counts)
    assert k.tolist() == [0, 1] and n.tolist() == [4, 2]
    assert np.allclose(c[0], [0.75, 1.5, 2.25], rtol=0, atol=1e-15)
    assert np.allclose(c[1], [4.0, 4.0, 4.0], rtol=0, atol=0)


def test_backward_matches_finite_differences():
    xyz = synth.rgbd_frame(96, 72, seed=6)
    leaf = 0.05
    d = oracle.downsample(xyz, leaf)
    V = len(d.keys)
    rng = np.random.Generator(np.random.PCG64(9))
    targets = d.centroids + rng.normal(size=d.centroids.shape) * 0.01
    grad_c = oracle.loss_grad_centroids(d.centroids, targets)
    grad = oracle.backward(grad_c, d.counts, d.point_to_voxel)
    assert (grad[d.point_to_voxel < 0] == 0).all()
    x64 = xyz.astype(np.float64)
    valid = _valid_rows(xyz)
    frac = np.zeros_like(x64)
    frac[valid] = (x64[valid] - d.origin.astype(np.float64)) / leaf - \
        _numpy_ijk(xyz[valid], d.origin, leaf)
    far = np.nonzero(valid & ((frac > 1e-3) & (frac < 1 - 1e-3)).all(axis=1))[0]
    pick = rng.choice(far, size=40, replace=False)
    h = 1e-4 * leaf
    for i in pick:
        for a in range(3):
            xp = x64.copy()
            xm = x64.copy()
            xp[i, a] += h
            xm[i, a] -= h
            lp = oracle.centroid_loss(xp, d.point_to_voxel, V, targets)
            lm = oracle.centroid_loss(xm, d.point_to_voxel, V, targets)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad[i, a]) <= 1e-3 * abs(grad[i, a]) + 1e-12


@pytest.mark.parametrize("leaf", [0.05, 0.02, 0.013])
def test_keys_near_faces_match_binary32(leaf):
    """Points within a few ulps of voxel faces: the key must be floor(fl(fl(p-o)/leaf)).

    Near a face, any other evaluation order (p/leaf - o/leaf, a reciprocal multiply,
    a fused multiply-add, double precision) gives a different voxel for some points.
    """
    rng = np.random.Generator(np.random.PCG64(21))
    o = rng.uniform(-3, 3, size=3).astype(np.float32)
    k = rng.integers(0, 400, size=(20000, 3))
    base = (o.astype(np.float64) + k * np.float64(leaf)).astype(np.float32)
    steps = rng.integers(-3, 4, size=(20000, 3))
    pts = base.copy()
    for s in range(1, 4):
        up = steps >= s
        dn = steps <= -s
        pts = np.where(up, np.nextafter(pts, np.float32(np.inf)), pts)
        pts = np.where(dn, np.nextafter(pts, np.float32(-np.inf)), pts)
    pts = pts.astype(np.float32)
    pts = pts[(pts >= o).all(axis=1)]
    keys, ijk, valid, st = oracle.keys(pts, o, leaf)
    assert st == 0 and valid.all()
    assert (ijk == _numpy_ijk(pts, o, leaf)).all()
    # the alternative order really differs on this set (the test has teeth)
    alt = np.floor(np.float32(pts) / np.float32(leaf) - o / np.float32(leaf)).astype(np.int64)
    assert (alt != ijk).any()
