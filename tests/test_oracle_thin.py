"""Pins of the oracle's reading R16: the paper's neighbour-count thinning loop (Sec. II-C,
Algorithm 1: 27-cell neighbour search with the Euclidean distance of Eq. 1, mark points
whose count exceeds the threshold, delete a batch of marked points per pass, delete the
rest of the marked points at the end), the random choice of the batch replaced by the
lowest given priorities."""
import numpy as np
import pytest

import oracle
from paper_2102_11084_gb300 import synth


def ranks(n, seed=0):
    return np.random.Generator(np.random.PCG64(seed)).permutation(n).astype(np.uint32)


@pytest.mark.parametrize("r_frac", [1.0, 0.6])
def test_counts_equal_all_pairs_brute_force(r_frac):
    x = synth.random_cloud(1500, seed=21, extent=0.5, nan_frac=0.0)
    cell = np.float32(0.05)
    o = x.min(axis=0)
    keys, ijk, valid, st = oracle.keys(x, o, float(cell))
    assert st == 0 and valid.all()
    r = np.float32(cell * np.float32(r_frac))
    alive = np.ones(x.shape[0], np.uint8)
    alive[::7] = 0
    got = oracle.neighbor_counts(x, ijk, alive, float(r))
    f = np.float32
    d = [(x[None, :, a] - x[:, None, a]).astype(f) for a in range(3)]
    d2 = ((d[0] * d[0]).astype(f) + (d[1] * d[1]).astype(f)).astype(f)
    d2 = (d2 + (d[2] * d[2]).astype(f)).astype(f)
    near = (d2 <= f(r * r)) & alive[None, :].astype(bool)
    np.fill_diagonal(near, False)
    want = np.where(alive.astype(bool), near.sum(axis=1), 0)
    assert np.array_equal(got, want)
    assert want.max() > 3  # the cloud is dense enough to matter


def clique_survivors(m, t, k):
    s = m
    while s > t + 1:  # every point of a clique of s has s - 1 neighbours
        s = s - k if s > k else 0
    return s


@pytest.mark.parametrize("m,t,k", [(10, 3, 2), (10, 3, 1000), (25, 4, 3), (25, 24, 5),
                                   (40, 0, 7), (7, 6, 1)])
def test_clique_closed_form(m, t, k):
    rng = np.random.Generator(np.random.PCG64(m * 100 + t))
    centre = np.float32([1.03, 2.07, 0.51])
    x = (centre + rng.uniform(-0.004, 0.004, size=(m, 3))).astype(np.float32)
    pr = ranks(m, seed=t)
    keep, passes, st = oracle.thin(x, 0.05, t, pr, batch=k)
    s = clique_survivors(m, t, k)
    assert st == 0 and keep.sum() == s
    if s:  # the lowest priorities went first
        assert set(np.nonzero(keep)[0]) == set(np.argsort(pr)[m - s:])


def test_sparse_or_permissive_clouds_are_untouched():
    g = np.stack(np.meshgrid(*[np.arange(6)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = (g * np.float32(0.3) + np.float32(0.01)).astype(np.float32)  # spacing 0.3 > r = 0.1
    keep, passes, _ = oracle.thin(x, 0.1, 0, ranks(x.shape[0]), batch=5)
    assert keep.all() and passes == 1
    y = synth.random_cloud(2000, seed=3, extent=0.3, nan_frac=0.1)
    keep, _, _ = oracle.thin(y, 0.05, 10 ** 6, ranks(2000), batch=10)
    assert np.array_equal(keep, np.isfinite(y).all(axis=1))


def test_invalid_points_dropped_and_range_reported():
    y = synth.random_cloud(500, seed=4, extent=0.3, nan_frac=0.2, inf_frac=0.05)
    keep, _, st = oracle.thin(y, 0.05, 5, ranks(500), batch=20)
    assert st == 0 and not keep[~np.isfinite(y).all(axis=1)].any()
    _, _, st = oracle.thin(np.float32([[0, 0, 0], [1e9, 0, 0]]), 1e-3, 1, ranks(2),
                           origin_xyz=np.zeros(3, np.float32))
    assert st == oracle.STATUS_RANGE


def test_a_point_exactly_at_distance_r_is_a_neighbour():
    # dyadic coordinates: d2 = r*r exactly, so "within r" decides by <=
    x = np.float32([[0.5, 0.5, 0.5], [0.75, 0.5, 0.5], [3.0, 3.0, 3.0]])
    keep, _, st = oracle.thin(x, 0.25, 0, ranks(3), batch=10, origin_xyz=np.zeros(3, np.float32))
    assert st == 0 and keep.tolist() == [False, False, True]
    keep, _, _ = oracle.thin(x, 0.25, 0, ranks(3), radius=0.2, batch=10,
                             origin_xyz=np.zeros(3, np.float32))
    assert keep.all()
