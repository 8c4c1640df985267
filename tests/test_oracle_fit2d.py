"""Pins of the oracle's 2D additive model and QuadTree initialisation (the
paper's 2D experiment, Sec. 3).

Render: the single-particle closed form with the FP32 support test replayed in
numpy float32; additivity over disjoint particle sets; order invariance.
Gradient: FP64 central differences (support far away), torch autograd of a
dense formulation with the same support mask. QuadTree: K = 1 is the image
mean; four constant quadrants give their colours; the leaves tile the image;
the greedy rule holds (every split cell's error is at least every splittable
leaf's, recomputed with numpy); the leaf count is 3m + 1 <= K. Densify/prune:
identity with the thresholds off; pruning keeps exactly the rows numpy selects;
a division gives four children centred on the parent on a square of side sigma
with half its scale and zero moments; the capacity divides the first
candidates."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_14244_gb300 import scenes


def _reach32(px, py, mx, my, D):
    f = np.float32
    dx = f(px) - f(mx)
    dy = f(py) - f(my)
    return f(f(dx * dx) + f(dy * dy)) < f(f(D) * f(D))


@pytest.mark.parametrize("D", [3.0, 7.5, 50.0])
def test_single_particle_closed_form(D):
    W, H = 37, 29
    p = np.array([[13.3, 11.7, np.log(4.2), 0.2, 0.5, 0.9, 0, 0]], np.float32)
    img = oracle.fit2d_render(p, D, W, H)
    s = float(np.exp(np.float64(p[0, 2])))
    for y in range(H):
        for x in range(W):
            px, py = np.float32(x + 0.5), np.float32(y + 0.5)
            if _reach32(px, py, p[0, 0], p[0, 1], D):
                d2 = (float(px) - float(p[0, 0])) ** 2 + (float(py) - float(p[0, 1])) ** 2
                want = p[0, 3:6].astype(np.float64) * np.exp(-d2 / (2 * s * s))
            else:
                want = np.zeros(3)
            np.testing.assert_allclose(img[:, y, x], want, rtol=1e-13, atol=1e-15)


def test_additive_and_order_invariant():
    p = scenes.fit2d_particles(60, 48, 1)
    a = oracle.fit2d_render(p[:25], 9.0, 48, 40)
    b = oracle.fit2d_render(p[25:], 9.0, 48, 40)
    ab = oracle.fit2d_render(p, 9.0, 48, 40)
    np.testing.assert_allclose(ab, a + b, rtol=1e-13, atol=1e-14)
    perm = np.random.default_rng(2).permutation(60)
    np.testing.assert_allclose(oracle.fit2d_render(p[perm], 9.0, 48, 40), ab, rtol=1e-13, atol=1e-14)


def _loss(p, D, Wt):
    return float((oracle.fit2d_render(p, D, Wt.shape[2], Wt.shape[1]) * Wt).sum())


def test_gradient_central_differences():
    # support far larger than the image: no pixel changes side under the steps
    p = scenes.fit2d_particles(6, 20, 3, sigma=(2.0, 6.0)).astype(np.float64)
    Wt = np.random.default_rng(4).normal(size=(3, 20, 22))
    g = oracle.fit2d_backward(p.astype(np.float32), 1000.0, Wt)
    assert np.all(g[:, 6:] == 0)
    for i in range(6):
        for j in range(6):
            h = 1e-3 if j < 2 else 1e-4
            pp, pm = p.copy(), p.copy()
            pp[i, j] += h
            pm[i, j] -= h
            # parameters move in FP32: use the rounded steps
            hp = float(np.float32(pp[i, j])) - float(np.float32(p[i, j]))
            hm = float(np.float32(p[i, j])) - float(np.float32(pm[i, j]))
            fd = (_loss(pp, 1000.0, Wt) - _loss(pm, 1000.0, Wt)) / (hp + hm)
            assert fd == pytest.approx(g[i, j], rel=2e-5, abs=1e-9), (i, j)


def test_gradient_matches_torch_autograd_with_cutoff():
    W, H, D = 40, 34, 8.0
    p32 = scenes.fit2d_particles(30, 36, 5, sigma=(1.5, 9.0))
    G = np.random.default_rng(6).normal(size=(3, H, W))
    g = oracle.fit2d_backward(p32, D, G)
    ys, xs = np.meshgrid(np.arange(H, dtype=np.float32) + np.float32(0.5),
                         np.arange(W, dtype=np.float32) + np.float32(0.5), indexing="ij")
    mask = np.stack([_reach32(xs, ys, p32[k, 0], p32[k, 1], D) for k in range(30)])   # [K][H][W]
    tp = torch.tensor(p32.astype(np.float64), requires_grad=True)
    tx, ty = torch.tensor(xs.astype(np.float64)), torch.tensor(ys.astype(np.float64))
    d2 = (tx[None] - tp[:, 0, None, None]) ** 2 + (ty[None] - tp[:, 1, None, None]) ** 2
    s = torch.exp(tp[:, 2])[:, None, None]
    gk = torch.exp(-d2 / (2 * s * s)) * torch.tensor(mask, dtype=torch.float64)
    img = torch.einsum("kc,khw->chw", tp[:, 3:6], gk)
    (img * torch.tensor(G)).sum().backward()
    np.testing.assert_allclose(img.detach().numpy(), oracle.fit2d_render(p32, D, W, H), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(g, tp.grad.numpy(), rtol=1e-10, atol=1e-12)


# ----------------------------------------------------------------- QuadTree --

def _quant(img):
    return np.rint(np.clip(img.astype(np.float64), 0, 1) * 4096)


def _cell_of(p):
    side = int(round(2 * np.exp(np.float64(p[2]))))
    return int(round(p[0] - side / 2)), int(round(p[1] - side / 2)), side


def test_quadtree_single_leaf_is_the_mean():
    img = scenes.fit2d_image(64, 7)
    p = oracle.quadtree_init(img, 1, 4)
    assert p.shape == (1, 8)
    assert tuple(p[0, :2]) == (32.0, 32.0)
    assert p[0, 2] == pytest.approx(np.log(32.0), rel=1e-7)
    np.testing.assert_allclose(p[0, 3:6], _quant(img).reshape(3, -1).mean(1) / 4096, rtol=1e-6)


def test_quadtree_constant_quadrants():
    img = np.zeros((3, 32, 32), np.float32)
    cols = np.array([[0.25, 0.5, 0.75], [1.0, 0.0, 0.5], [0.125, 0.875, 0.375], [0.625, 0.25, 1.0]], np.float32)
    for j, (y0, x0) in enumerate(((0, 0), (0, 16), (16, 0), (16, 16))):
        img[:, y0:y0 + 16, x0:x0 + 16] = cols[j][:, None, None]
    p = oracle.quadtree_init(img, 4, 2)
    assert p.shape == (4, 8)
    np.testing.assert_array_equal(p[:, :2], [[8, 8], [24, 8], [8, 24], [24, 24]])
    np.testing.assert_array_equal(p[:, 3:6], cols)
    np.testing.assert_allclose(np.exp(p[:, 2].astype(np.float64)), 8.0, rtol=1e-7)
    # a further split budget finds nothing to gain but still splits (all errors are 0): ties by level, row, column
    p7 = oracle.quadtree_init(img, 7, 2)
    assert p7.shape == (7, 8) and _cell_of(p7[0]) == (16, 0, 16)


@pytest.mark.parametrize("k,min_cell", [(100, 2), (334, 4), (1000, 1), (40, 16)])
def test_quadtree_tiles_the_image_and_is_greedy(k, min_cell):
    S = 64
    img = scenes.fit2d_image(S, 8)
    p = oracle.quadtree_init(img, k, min_cell)
    L = p.shape[0]
    assert L <= k and (L - 1) % 3 == 0
    cover = np.zeros((S, S), int)
    cells = [_cell_of(q) for q in p]
    for x0, y0, side in cells:
        cover[y0:y0 + side, x0:x0 + side] += 1
        assert side >= min_cell
    assert np.all(cover == 1)
    q = _quant(img)

    def err(x0, y0, side):  # SSE of the quantised cell, summed over channels (numpy)
        blk = q[:, y0:y0 + side, x0:x0 + side].reshape(3, -1)
        return float(((blk - blk.mean(1, keepdims=True)) ** 2).sum())

    # the split cells are the ancestors of the leaves
    split = set()
    for x0, y0, side in cells:
        s = side
        while s < S:
            s *= 2
            split.add((x0 // s * s, y0 // s * s, s))
    leaf_err = [err(*c) for c in cells if c[2] // 2 >= min_cell]
    if leaf_err and L + 3 <= k:
        pytest.fail("budget left but a splittable leaf was not split")
    worst_split = min(err(*c) for c in split) if split else np.inf
    if leaf_err:
        assert worst_split >= max(leaf_err) * (1 - 1e-12)
    # each particle's colour is its cell's mean of the quantised image
    for (x0, y0, side), pp in zip(cells, p):
        np.testing.assert_allclose(pp[3:6], q[:, y0:y0 + side, x0:x0 + side].reshape(3, -1).mean(1) / 4096,
                                   rtol=1e-6)


def test_quadtree_rejects_bad_sizes():
    with pytest.raises(ValueError):
        oracle.quadtree_init(np.zeros((3, 48, 48), np.float32), 10, 2)
    with pytest.raises(ValueError):
        oracle.quadtree_init(np.zeros((3, 1024, 1024), np.float32), 10, 2)


# ------------------------------------------------------------ densify/prune --

def _moments(k, seed):
    rng = np.random.default_rng(seed)
    return rng.random((k, 8)).astype(np.float32), rng.random((k, 8)).astype(np.float32)


def test_densify_thresholds_off_is_identity():
    p = scenes.fit2d_particles(50, 64, 11)
    m, v = _moments(50, 12)
    acc = np.random.default_rng(13).random(50).astype(np.float32)
    q, qm, qv = oracle.fit2d_densify(p, m, v, acc, 10, 0.0, np.inf, -np.inf, 200)
    np.testing.assert_array_equal(q, p)
    np.testing.assert_array_equal(qm, m)
    np.testing.assert_array_equal(qv, v)


def test_densify_prunes_small_amplitudes():
    p = scenes.fit2d_particles(200, 64, 14)
    p[::3, 3:6] *= 0.01
    p[1::7, 4] = -0.5                  # |A| counts, not A
    m, v = _moments(200, 15)
    acc = np.zeros(200, np.float32)
    tau = 0.05
    keep = np.abs(p[:, 3:6]).max(1) >= tau
    q, qm, qv = oracle.fit2d_densify(p, m, v, acc, 1, tau, np.inf, 0.0, 200)
    np.testing.assert_array_equal(q, p[keep])
    np.testing.assert_array_equal(qm, m[keep])
    np.testing.assert_array_equal(qv, v[keep])


def test_densify_divides_into_four_half_size_children():
    p = scenes.fit2d_particles(40, 64, 16, sigma=(1.0, 8.0))
    m, v = _moments(40, 17)
    acc = np.random.default_rng(18).random(40).astype(np.float32)
    n_it, tau_g, lsm = 4, 0.1, float(np.log(2.0))
    cand = (acc > np.float32(tau_g) * np.float32(n_it)) & (p[:, 2] >= np.float32(lsm))
    q, qm, qv = oracle.fit2d_densify(p, m, v, acc, n_it, 0.0, tau_g, lsm, 1000)
    assert q.shape[0] == 40 + 3 * cand.sum()
    o = 0
    for i in range(40):
        if not cand[i]:
            np.testing.assert_array_equal(q[o], p[i])
            np.testing.assert_array_equal(qm[o], m[i])
            o += 1
            continue
        kids = q[o:o + 4]
        s = np.exp(np.float64(p[i, 2]))
        np.testing.assert_allclose(kids[:, :2].mean(0), p[i, :2], rtol=1e-6, atol=1e-5)    # centred on the parent
        np.testing.assert_allclose(np.ptp(kids[:, 0]), s, rtol=1e-5)                       # a square of side sigma
        np.testing.assert_allclose(np.ptp(kids[:, 1]), s, rtol=1e-5)
        np.testing.assert_allclose(np.exp(kids[:, 2].astype(np.float64)), s / 2, rtol=1e-6)  # half the scale
        np.testing.assert_array_equal(kids[:, 3:6], np.repeat(p[i:i + 1, 3:6], 4, 0))
        assert np.all(qm[o:o + 4] == 0) and np.all(qv[o:o + 4] == 0)
        o += 4
    assert o == q.shape[0]


def test_densify_capacity_divides_the_first_candidates():
    p = scenes.fit2d_particles(30, 64, 19, sigma=(2.0, 8.0))
    m, v = _moments(30, 20)
    acc = np.full(30, 10.0, np.float32)
    q, _, _ = oracle.fit2d_densify(p, m, v, acc, 1, 0.0, 1.0, -np.inf, 30 + 3 * 5 + 2)
    assert q.shape[0] == 45
    # the first five parents divided: their children come first, then the rest unchanged
    np.testing.assert_array_equal(q[20:], p[5:])
    for i in range(5):
        np.testing.assert_allclose(q[4 * i:4 * i + 4, :2].mean(0), p[i, :2], rtol=1e-6, atol=1e-5)


def test_densify_capacity_below_kept_count_truncates():
    p = scenes.fit2d_particles(30, 64, 21)
    m, v = _moments(30, 22)
    acc = np.full(30, 10.0, np.float32)
    q, qm, _ = oracle.fit2d_densify(p, m, v, acc, 1, 0.0, 1.0, -np.inf, 12)
    # no room to divide anything: the first 12 particles, unchanged
    np.testing.assert_array_equal(q, p[:12])
    np.testing.assert_array_equal(qm, m[:12])


def test_grad_accum_is_the_fp32_norm_sum():
    g = np.zeros((4, 8), np.float32)
    g[0, :2] = (3.0, 4.0)              # a 3-4-5 triangle: exactly 5
    g[1, :2] = (-6.0, 8.0)             # signs do not matter: 10
    g[2, 2:] = 7.0                     # other slots do not count
    acc = oracle.fit2d_grad_accum(g, np.array([1.0, 0.5, 2.0, 0.0], np.float32))
    np.testing.assert_array_equal(acc, np.array([6.0, 10.5, 2.0, 0.0], np.float32))
    rng = np.random.default_rng(23)
    g = rng.normal(size=(1000, 8)).astype(np.float32)
    a0 = rng.random(1000).astype(np.float32)
    want = a0 + np.sqrt(g[:, 0] * g[:, 0] + g[:, 1] * g[:, 1])    # numpy float32: one rounding per step
    np.testing.assert_array_equal(oracle.fit2d_grad_accum(g, a0), want)
    assert np.allclose(want, a0 + np.hypot(g[:, 0].astype(np.float64), g[:, 1]), rtol=1e-6)
