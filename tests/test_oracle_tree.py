"""Pins of the oracle's Morton keys, sort and adaptive octree.

The tree is the paper's adaptive tree with N_crit the maximum number of
particles per cell (Results section); quantisation and key layout are the
readings R1/R2 stated in the oracle's header."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_5815_gb300 import inputs
from tests.oracle_helpers import cell_index

SPREAD_ALL = int("".join("001" for _ in range(21)), 2)  # bits 0,3,...,60


def test_keys_of_hand_computed_points():
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [0.5, 0.25, 0]], float)
    lo, side, keys = O.morton_keys(x)
    assert np.array_equal(lo, [0, 0, 0]) and side == 1.0
    # a coordinate at the maximum face is clamped to cell 2^21 - 1
    assert int(keys[0]) == 0
    assert int(keys[1]) == SPREAD_ALL
    assert int(keys[2]) == SPREAD_ALL << 1
    assert int(keys[3]) == SPREAD_ALL << 2
    assert int(keys[4]) == (1 << 63) - 1
    # 0.5 -> k_x = 2^20 (key bit 60); 0.25 -> k_y = 2^19 (key bit 3*19+1 = 58)
    assert int(keys[5]) == (1 << 60) | (1 << 58)


def test_box_is_cube_on_largest_extent():
    x = np.array([[1.0, 2.0, 3.0], [1.5, 6.0, 3.25]])
    lo, side, keys = O.morton_keys(x)
    assert np.array_equal(lo, [1.0, 2.0, 3.0]) and side == 4.0
    # second point: x: 0.5/4*2^21 = 2^18, y: clamp, z: 0.25/4*2^21 = 2^17
    k = cell_index(np.array([21]), keys[1:2])[0]
    assert list(k) == [1 << 18, (1 << 21) - 1, 1 << 17]


def test_nonfinite_rejected():
    x = np.array([[0.0, 0.0, 0.0], [np.nan, 1.0, 0.0]])
    with pytest.raises(ValueError):
        O.morton_keys(x)
    with pytest.raises(ValueError):
        O.Fmm(x, np.ones(2), 4, 0.5, 4)


@pytest.mark.parametrize("dist,n,ncrit,max_depth", [("uniform", 3000, 16, 21),
                                                     ("plummer", 3000, 8, 21),
                                                     ("plummer", 3000, 8, 4)])
def test_tree_invariants_and_containment(dist, n, ncrit, max_depth):
    x, q = inputs.make(dist, n, 11)
    f = O.Fmm(x, q, 3, 0.5, ncrit, max_depth=max_depth)
    key, order = f.sorted()
    assert np.array_equal(np.sort(order), np.arange(n))
    # sorted by (key, original index)
    assert np.all((key[1:] > key[:-1]) | ((key[1:] == key[:-1]) & (order[1:] > order[:-1])))
    c = f.cells()
    cnt = c["end"] - c["begin"]
    assert np.all(cnt > 0)
    leaf = c["nchild"] == 0
    assert np.all(cnt[~leaf] > ncrit) and np.all(c["level"][~leaf] < max_depth)
    assert np.all((cnt[leaf] <= ncrit) | (c["level"][leaf] == max_depth))
    # every particle in exactly one leaf
    mark = np.zeros(n, int)
    for b, e in zip(c["begin"][leaf], c["end"][leaf]):
        mark[b:e] += 1
    assert np.all(mark == 1)
    # children partition the parent's range, in octant order
    for ci in np.flatnonzero(~leaf):
        kids = np.flatnonzero(c["parent"] == ci)
        assert c["begin"][kids[0]] == c["begin"][ci] and c["end"][kids[-1]] == c["end"][ci]
        assert np.all(c["begin"][kids[1:]] == c["end"][kids[:-1]])
        assert np.all(np.diff(c["prefix"][kids] & np.uint64(7)).astype(np.int64) > 0)
    # geometric containment: each particle lies in its leaf's box
    lo, side = f.box()
    xs = x.astype(np.float64)[order]
    k = cell_index(c["level"], c["prefix"])
    for ci in np.flatnonzero(leaf):
        w = side / 2.0 ** c["level"][ci]
        lo_c = lo + k[ci] * w
        pts = xs[c["begin"][ci]:c["end"][ci]]
        assert np.all(pts >= lo_c - 1e-12 * side) and np.all(pts <= lo_c + w + 1e-12 * side)


def test_identical_points_make_a_chain():
    x = np.tile(np.array([[0.3, 0.3, 0.3]], np.float32), (10, 1))
    f = O.Fmm(x, np.ones(10), 3, 0.5, 4, max_depth=6)
    c = f.cells()
    assert f.ncells == 7 and f.depth == 6
    assert np.all(c["end"] - c["begin"] == 10)
    phi, g = f.evaluate()
    assert np.all(phi == 0) and np.all(g == 0)


def test_root_is_leaf_when_ncrit_covers_everything():
    x, q = inputs.uniform_cube(50, 5)
    f = O.Fmm(x, q, 4, 0.5, 50)
    assert f.ncells == 1 and f.nm2l == 0 and f.np2p == 1
    phi, g = f.evaluate()
    pd, gd = O.direct(x, q)
    assert np.allclose(phi, pd, rtol=1e-13) and np.allclose(g, gd, rtol=1e-12)
