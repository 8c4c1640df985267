"""Pins of the oracle's Octree initialisation of 3D Gaussians (Sec. 3.1: an
Octree for 3D, colour = the cell average, sigma = half the cell width) from a
coloured point set: one leaf = the whole cube with the numpy mean colour; eight
constant octants split into their eight colours; the leaves partition the
points (membership recomputed with numpy's FP32 cell index) and each colour is
its cell's 12-bit mean; the greedy rule (every split cell's error >= every
splittable leaf's, recomputed in numpy; the budget respected and exhausted);
parameterisations; SH DC; non-finite and outside points."""
import numpy as np
import pytest

import oracle


def _cloud(n, seed, lo=(-1.0, -1.0, -1.0), side=2.0):
    rng = np.random.default_rng(seed)
    p = (np.asarray(lo) + side * rng.random((n, 3))).astype(np.float32)
    # colour fields with structure at several scales
    c = np.stack([0.5 + 0.4 * np.sin(3 * p[:, 0]), 0.5 + 0.4 * np.cos(5 * p[:, 1] * p[:, 2]),
                  (p[:, 2] > 0.3).astype(np.float64) * 0.8 + 0.1], 1)
    c = np.clip(c + rng.normal(0, 0.02, c.shape), 0, 1).astype(np.float32)
    return p, c


def _q(c):
    return np.rint(np.clip(c, 0, 1).astype(np.float32) * np.float32(4096)).astype(np.int64)


def _cell_index(p, lo, side, L):
    inv = np.float32((1 << L) / side)
    t = np.floor((p - np.asarray(lo, np.float32)) * inv)
    return np.clip(t, 0, (1 << L) - 1).astype(np.int64)


def _leaves(ms, lo, side, L):
    """(level, cell coordinates) of each emitted Gaussian, from its centre and sigma."""
    lv = np.rint(np.log2(side / (2 * ms[:, 3].astype(np.float64)))).astype(int)
    cs = side / (1 << lv)
    ij = np.floor((ms[:, :3].astype(np.float64) - np.asarray(lo)) / cs[:, None]).astype(np.int64)
    return lv, ij


def test_single_leaf_is_the_cube_mean():
    p, c = _cloud(3000, 1)
    ms, op, col = oracle.octree_init(p, c, (-1, -1, -1), 2.0, 5, 1, opacity=0.3)
    assert ms.shape == (1, 4)
    np.testing.assert_allclose(ms[0], [0, 0, 0, 1.0], atol=1e-7)
    np.testing.assert_allclose(col[0], _q(c).mean(0) / 4096.0, rtol=1e-6)
    assert op[0] == np.float32(0.3)


def test_eight_constant_octants():
    rng = np.random.default_rng(2)
    p = rng.uniform(-0.99, 0.99, (4000, 3)).astype(np.float32)
    octant = (p[:, 0] > 0).astype(int) | ((p[:, 1] > 0).astype(int) << 1) | ((p[:, 2] > 0).astype(int) << 2)
    colours = rng.random((8, 3)).astype(np.float32)
    c = colours[octant]
    ms, _, col = oracle.octree_init(p, c, (-1, -1, -1), 2.0, 4, 8)
    assert ms.shape[0] == 8                           # the root splits once, the octants are exact
    for k in range(8):                                # Morton order: x lowest bit
        want = np.array([(k & 1) - 0.5, ((k >> 1) & 1) - 0.5, ((k >> 2) & 1) - 0.5, 0.5], np.float32)
        np.testing.assert_allclose(ms[k], want, atol=1e-7)
        np.testing.assert_allclose(col[k], _q(colours[k:k + 1])[0] / 4096.0, rtol=1e-6)


@pytest.mark.parametrize("k_max,L", [(50, 4), (400, 5), (2000, 6)])
def test_leaves_partition_points_and_greedy_rule(k_max, L):
    lo, side = (-1.0, -1.0, -1.0), 2.0
    p, c = _cloud(20000, 3 + k_max, lo, side)
    ms, _, col = oracle.octree_init(p, c, lo, side, L, k_max)
    K = ms.shape[0]
    assert 1 <= K <= k_max
    lv, ij = _leaves(ms, lo, side, L)
    fine = _cell_index(p, lo, side, L)
    owner = -np.ones(len(p), int)
    for k in range(K):
        inside = np.all((fine >> (L - lv[k])) == ij[k], axis=1)
        assert np.all(owner[inside] == -1)             # no point in two leaves
        owner[inside] = k
        assert inside.any()                           # only non-empty leaves
        np.testing.assert_allclose(col[k], _q(c[inside]).mean(0) / 4096.0, rtol=1e-6)
    assert np.all(owner >= 0)                         # every point in a leaf

    def err(mask):
        q = _q(c[mask])
        n = float(mask.sum())
        return max(0.0, float(sum(float((q[:, ch] ** 2).sum()) - float(q[:, ch].sum()) ** 2 / n for ch in range(3))))

    # the cells that were split: every ancestor of a leaf
    split = set()
    for k in range(K):
        for l in range(lv[k]):
            split.add((l, tuple(ij[k] >> (lv[k] - l))))
    split_err = [err(np.all((fine >> (L - l)) == np.array(x), axis=1)) for l, x in split]
    leaf_err, leaf_kids = [], []
    for k in range(K):
        inside = owner == k
        if lv[k] < L and inside.sum() >= 2:
            leaf_err.append(err(inside))
            sub = (fine[inside] >> (L - lv[k] - 1))
            leaf_kids.append(len({tuple(r) for r in sub}))
    if split_err and leaf_err:
        assert min(split_err) >= max(leaf_err) - 1e-6 * max(1.0, max(leaf_err))
    if leaf_err:                                      # the next split (first in the order) did not fit
        nxt = int(np.argmax(leaf_err))
        assert K + leaf_kids[nxt] - 1 > k_max


def test_log_parameters_and_sh_dc():
    p, c = _cloud(5000, 9)
    ms0, op0, col0 = oracle.octree_init(p, c, (-1, -1, -1), 2.0, 5, 60, opacity=0.25)
    ms1, op1, col1 = oracle.octree_init(p, c, (-1, -1, -1), 2.0, 5, 60, opacity=0.25, sh_degree=3, param_mode=1)
    np.testing.assert_array_equal(ms0[:, :3], ms1[:, :3])
    np.testing.assert_allclose(np.exp(ms1[:, 3].astype(np.float64)), ms0[:, 3], rtol=1e-6)
    np.testing.assert_allclose(1 / (1 + np.exp(-op1.astype(np.float64))), 0.25, rtol=1e-6)
    y00 = 1.0 / (2.0 * np.sqrt(np.pi))
    assert col1.shape[1] == 48
    np.testing.assert_allclose(col1[:, :3].astype(np.float64) * y00 + 0.5, col0, rtol=1e-5, atol=1e-6)
    assert np.all(col1[:, 3:] == 0)


def test_nonfinite_ignored_outside_clamped():
    p, c = _cloud(1000, 10)
    p2 = np.concatenate([p, [[np.nan, 0, 0], [0, np.inf, 0], [5, 5, 5], [-7, 0.1, 0.2]]]).astype(np.float32)
    c2 = np.concatenate([c, np.full((4, 3), 0.9, np.float32)]).astype(np.float32)
    ms, _, col = oracle.octree_init(p2, c2, (-1, -1, -1), 2.0, 3, 1)
    want = _q(np.concatenate([c, c2[-2:]])).mean(0) / 4096.0      # the two finite outliers count, clamped in
    np.testing.assert_allclose(col[0], want, rtol=1e-6)


def test_property_checker_accepts_the_oracle_and_catches_mistakes():
    """The vectorised checker used at full size on the GPU (tests/_octree_props.py) accepts the
    oracle's trees and rejects planted mistakes: a missing leaf, a colour one ulp off, two leaves
    swapped, a tree grown with a smaller budget, a leaf's centre moved, and a tree grown from other
    colours (the same colours on other points) but given its cells' true means, which only the
    order of the splits gives away."""
    from tests._octree_props import check_octree
    lo, side, L = (-1.0, -1.0, -1.0), 2.0, 6
    p, c = _cloud(30000, 21, lo, side)
    for k_max in (1, 9, 300, 2500):
        ms, op, col = oracle.octree_init(p, c, lo, side, L, k_max, opacity=0.4)
        check_octree(p, c, lo, side, L, k_max, ms, op, col, 0.4)
    ms, op, col = oracle.octree_init(p, c, lo, side, L, 2500, opacity=0.4)
    bad = [
        (ms[:-1], op[:-1], col[:-1], 2500),
        (ms, op, np.where(np.arange(len(col))[:, None] == 7, np.nextafter(col, np.float32(2)), col), 2500),
        (ms[[1, 0] + list(range(2, len(ms)))], op, col[[1, 0] + list(range(2, len(col)))], 2500),
    ]
    ms2, op2, col2 = oracle.octree_init(p, c, lo, side, L, 2000, opacity=0.4)
    bad.append((ms2, op2, col2, 2500))
    moved = ms.copy()
    moved[5, 0] = np.nextafter(moved[5, 0], np.float32(9))
    bad.append((moved, op, col, 2500))
    other = np.ascontiguousarray(c[np.random.default_rng(5).permutation(len(c))])
    ms3, op3, _ = oracle.octree_init(p, other, lo, side, L, 2500, opacity=0.4)
    lv, ij = _leaves(ms3, lo, side, L)
    fine = _cell_index(p, lo, side, L)
    col3 = np.stack([(_q(c[np.all((fine >> (L - lv[k])) == ij[k], axis=1)]).sum(0) /
                      (4096.0 * np.all((fine >> (L - lv[k])) == ij[k], axis=1).sum())).astype(np.float32)
                     for k in range(len(ms3))])
    bad.append((ms3, op3, col3, 2500))
    for m_, o_, c_, k_ in bad:
        with pytest.raises(AssertionError):
            check_octree(p, c, lo, side, L, k_, m_, o_, c_, 0.4)


@pytest.mark.parametrize("k_max", [64, 200, 1000])
def test_property_checker_accepts_ties(k_max):
    """Colours constant on the 64 level-2 cells (every finer cell has error 0): the oracle's trees
    end inside a run of equal keys, and the checker's id order among equal keys accepts them."""
    from tests._octree_props import check_octree
    rng = np.random.default_rng(11)
    p = rng.uniform(-1, 1, (20000, 3)).astype(np.float32)
    cell = np.clip(np.floor((p + 1) * 2), 0, 3).astype(np.int64)
    c = rng.uniform(0, 1, (64, 3)).astype(np.float32)[cell[:, 0] + 4 * cell[:, 1] + 16 * cell[:, 2]]
    lo, side, L = (-1.0, -1.0, -1.0), 2.0, 5
    ms, op, col = oracle.octree_init(p, c, lo, side, L, k_max, opacity=0.4)
    check_octree(p, c, lo, side, L, k_max, ms, op, col, 0.4)
