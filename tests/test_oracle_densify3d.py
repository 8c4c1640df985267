"""Pins of the oracle's densify / prune of the 3D Gaussians (Sec. 3.2: deletion
below a threshold, division; Sec. 2.5; the Octree of Sec. 3.1 as the division
pattern) against numpy recomputations of each rule: identity with the rules off,
pruning as a numpy selection, the candidate rule, the eight children's geometry
(centred on the parent, one per octant at +- sigma / 2, half the scale, same
opacity and colour, zero moments), the capacity rule, and the statistic."""
import numpy as np
import pytest

import oracle

C = 48


def _state(n, seed, param_mode=1):
    rng = np.random.default_rng(seed)
    ms = np.zeros((n, 4), np.float32)
    ms[:, :3] = rng.uniform(-1, 1, (n, 3))
    sig = np.exp(rng.uniform(np.log(0.005), np.log(0.05), n))
    ms[:, 3] = np.log(sig) if param_mode == 1 else sig
    op = (rng.normal(0, 1.5, n) if param_mode == 1 else rng.uniform(0.01, 0.95, n)).astype(np.float32)
    col = rng.normal(0, 0.3, (n, C)).astype(np.float32)
    m = [rng.normal(0, 1e-3, a.shape).astype(np.float32) for a in (ms, op, col)]
    v = [rng.random(a.shape).astype(np.float32) * np.float32(1e-6) for a in (ms, op, col)]
    acc = rng.random(n).astype(np.float32) * np.float32(4.0)
    vis = rng.integers(0, 5, n).astype(np.uint32)
    return (ms, op, col), m, v, acc, vis


def test_rules_off_is_identity():
    p, m, v, acc, vis = _state(300, 1)
    q, qm, qv = oracle.densify3d(p, m, v, acc, vis, 1, -np.inf, np.inf, -np.inf, 1000)
    for a, b in zip(q + qm + qv, p + tuple(m) + tuple(v)):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("param_mode", [0, 1])
def test_prune_is_a_selection_by_opacity(param_mode):
    p, m, v, acc, vis = _state(400, 2, param_mode)
    op_min = np.float32(0.0 if param_mode == 1 else 0.3)
    keep = p[1] >= op_min
    q, qm, qv = oracle.densify3d(p, m, v, acc, vis, param_mode, op_min, np.inf, -np.inf, 1000)
    for a, b in zip(q + qm + qv, p + tuple(m) + tuple(v)):
        np.testing.assert_array_equal(a, b[keep])


@pytest.mark.parametrize("param_mode", [0, 1])
def test_division_into_eight_octant_children(param_mode):
    p, m, v, acc, vis = _state(120, 3, param_mode)
    tau_g = np.float32(0.9)
    smin = np.float32(np.log(0.01) if param_mode == 1 else 0.01)
    cand = (vis > 0) & (acc > tau_g * vis.astype(np.float32)) & (p[0][:, 3] >= smin)
    assert 0 < cand.sum() < 120
    q, qm, qv = oracle.densify3d(p, m, v, acc, vis, param_mode, -np.inf, tau_g, smin, 10000)
    assert q[0].shape[0] == 120 + 7 * cand.sum()
    o = 0
    for i in range(120):
        if not cand[i]:
            for a, b in zip((q[0][o], q[1][o], q[2][o], qm[2][o]), (p[0][i], p[1][i], p[2][i], m[2][i])):
                np.testing.assert_array_equal(a, b)
            o += 1
            continue
        kids = q[0][o:o + 8]
        s = np.float64(p[0][i, 3])
        sigma = np.exp(s) if param_mode == 1 else s
        off = kids[:, :3].astype(np.float64) - p[0][i, :3]
        np.testing.assert_allclose(np.abs(off), sigma / 2, rtol=1e-4, atol=1e-7)       # +- sigma / 2 per axis
        signs = (off > 0).astype(int)
        assert sorted((signs * [1, 2, 4]).sum(1).tolist()) == list(range(8))          # one child per octant
        np.testing.assert_allclose(kids[:, :3].mean(0), p[0][i, :3], atol=1e-6)        # centred on the parent
        child = np.exp(kids[:, 3].astype(np.float64)) if param_mode == 1 else kids[:, 3]
        np.testing.assert_allclose(child, sigma / 2, rtol=1e-6)                        # half the scale
        np.testing.assert_array_equal(q[1][o:o + 8], np.full(8, p[1][i]))
        np.testing.assert_array_equal(q[2][o:o + 8], np.repeat(p[2][i:i + 1], 8, 0))
        for a in qm + qv:
            assert np.all(a[o:o + 8] == 0)
        o += 8
    assert o == q[0].shape[0]


def test_unseen_gaussians_never_divide():
    p, m, v, acc, vis = _state(50, 4)
    vis[:] = 0
    q, _, _ = oracle.densify3d(p, m, v, acc, vis, 1, -np.inf, 0.0, -np.inf, 1000)
    np.testing.assert_array_equal(q[0], p[0])


def test_capacity_divides_the_first_candidates():
    p, m, v, acc, vis = _state(40, 5)
    acc[:] = 10.0
    vis[:] = 1
    q, _, _ = oracle.densify3d(p, m, v, acc, vis, 1, -np.inf, 1.0, -np.inf, 40 + 7 * 3 + 5)
    assert q[0].shape[0] == 61
    np.testing.assert_array_equal(q[0][24:], p[0][3:])          # three divided, the rest kept
    for i in range(3):
        np.testing.assert_allclose(q[0][8 * i:8 * i + 8, :3].mean(0), p[0][i, :3], atol=1e-6)
    q, _, _ = oracle.densify3d(p, m, v, acc, vis, 1, -np.inf, 1.0, -np.inf, 25)
    np.testing.assert_array_equal(q[0], p[0][:25])               # no room: the first 25 kept


def test_grad_accum3d_matches_numpy_float32():
    rng = np.random.default_rng(6)
    n = 2000
    g = rng.normal(size=(n, 8)).astype(np.float32)
    cnt = rng.integers(0, 3, n).astype(np.uint32)
    a0 = rng.random(n).astype(np.float32)
    v0 = rng.integers(0, 9, n).astype(np.uint32)
    acc, vis = oracle.grad_accum3d(g, cnt, a0, v0)
    seen = cnt > 0
    want = np.where(seen, a0 + np.sqrt(g[:, 0] * g[:, 0] + g[:, 1] * g[:, 1]), a0)
    np.testing.assert_array_equal(acc, want)
    np.testing.assert_array_equal(vis, v0 + seen.astype(np.uint32))
    g[:2, :2] = [[3.0, 4.0], [0.0, -2.0]]
    acc, _ = oracle.grad_accum3d(g[:2], np.ones(2, np.uint32), np.zeros(2, np.float32), np.zeros(2, np.uint32))
    np.testing.assert_array_equal(acc, [5.0, 2.0])
