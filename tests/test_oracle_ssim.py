"""Pins of the oracle's structural term of the loss of Sec. 3,
L = (1 - lambda) |f - f^|_1 + lambda (1 - SSIM).

The window and its zero padding are pinned by scipy's gaussian_filter (a
library routine) and by closed forms on constant images; SSIM(x, x) = 1 with a
zero gradient; symmetry; lambda = 0 reduces to the (pinned) L1 term; the
analytic gradient against FP64 central differences and against torch's
autograd through conv2d (library routines)."""
import numpy as np
import pytest
import torch
from scipy.ndimage import gaussian_filter

import oracle

C1, C2 = 0.01 ** 2, 0.03 ** 2


def _gf(a):
    # radius int(truncate * sigma + 0.5) = 5, weights exp(-k^2 / (2 sigma^2)) normalised, zeros outside
    return gaussian_filter(a, sigma=1.5, mode="constant", cval=0.0, truncate=5.0 / 1.5)


def _images(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.random(shape), rng.random(shape)


def test_identical_images_give_one_and_zero_gradient():
    x, _ = _images((3, 21, 18), 1)
    loss, ssim, g, smap = oracle.l1_ssim(x, x, lam=1.0, ssim_map=True)
    assert np.all(np.abs(smap - 1.0) < 1e-13)
    assert abs(ssim - 1.0) < 1e-13 and abs(loss) < 1e-13
    assert np.abs(g).max() < 1e-15


@pytest.mark.parametrize("a,b", [(0.3, 0.7), (0.9, 0.05), (0.5, 0.5), (0.0, 0.2)])
def test_constant_images_closed_form(a, b):
    H, W = 23, 19
    x, y = np.full((1, H, W), a), np.full((1, H, W), b)
    _, _, _, smap = oracle.l1_ssim(x, y, grad=False, ssim_map=True)
    s = _gf(np.ones((H, W)))          # in-image part of the window at each pixel
    mx, my = a * s, b * s
    sxx, syy, sxy = a * a * (s - s * s), b * b * (s - s * s), a * b * (s - s * s)
    ref = (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    np.testing.assert_allclose(smap[0], ref, rtol=1e-12, atol=1e-14)
    inner = smap[0, 5:-5, 5:-5]
    np.testing.assert_allclose(inner, (2 * a * b + C1) / (a * a + b * b + C1), rtol=1e-12)


def test_window_means_match_gaussian_filter():
    x, y = _images((2, 30, 27), 2)
    _, ssim, _, smap = oracle.l1_ssim(x, y, grad=False, ssim_map=True)
    for c in range(2):
        mx, my = _gf(x[c]), _gf(y[c])
        sxx, syy, sxy = _gf(x[c] * x[c]) - mx * mx, _gf(y[c] * y[c]) - my * my, _gf(x[c] * y[c]) - mx * my
        ref = (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
        np.testing.assert_allclose(smap[c], ref, rtol=1e-11, atol=1e-13)
    assert abs(ssim - smap.mean()) < 1e-14


def test_symmetric_and_bounded():
    x, y = _images((3, 16, 40), 3)
    _, s1, _, m1 = oracle.l1_ssim(x, y, grad=False, ssim_map=True)
    _, s2, _, m2 = oracle.l1_ssim(y, x, grad=False, ssim_map=True)
    np.testing.assert_allclose(m1, m2, rtol=1e-12, atol=1e-13)
    assert np.all(m1 <= 1.0) and np.all(m1 >= -1.0)
    # more noise, less similarity (same noise pattern, growing amplitude)
    n = np.random.default_rng(4).normal(size=x.shape)
    vals = [oracle.l1_ssim(x, x + e * n, grad=False)[1] for e in (0.01, 0.05, 0.2, 0.5)]
    assert all(a > b for a, b in zip(vals, vals[1:]))


def test_lambda_zero_is_the_l1_term():
    x, y = _images((3, 12, 13), 5)
    y = y.astype(np.float32).astype(np.float64)   # the L1 oracle takes an FP32 target
    loss, _, g = oracle.l1_ssim(x, y, lam=0.0)
    l1, g1 = oracle.l1(x, y)
    assert loss == pytest.approx(l1, rel=1e-14)
    np.testing.assert_array_equal(g, g1)


def test_gradient_central_differences():
    x, y = _images((2, 9, 8), 6)
    lam = 0.2
    _, _, g = oracle.l1_ssim(x, y, lam=lam)
    rng = np.random.default_rng(7)
    idx = [tuple(rng.integers(0, s) for s in x.shape) for _ in range(40)]
    for k in idx:
        # keep the L1 kink away: |x - y| well above h
        if abs(x[k] - y[k]) < 1e-3:
            continue
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[k] += h
        xm[k] -= h
        fd = (oracle.l1_ssim(xp, y, lam=lam, grad=False)[0] - oracle.l1_ssim(xm, y, lam=lam, grad=False)[0]) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-6, abs=1e-11)


def test_gradient_matches_torch_autograd():
    x, y = _images((3, 14, 11), 8)
    lam = 0.2
    loss, ssim, g = oracle.l1_ssim(x, y, lam=lam)
    k = torch.arange(-5, 6, dtype=torch.float64)
    w2 = torch.exp(-(k[:, None] ** 2 + k[None, :] ** 2) / (2 * 1.5 ** 2))
    w2 = (w2 / w2.sum()).expand(3, 1, 11, 11)
    tx = torch.tensor(x, requires_grad=True)
    ty = torch.tensor(y)

    def filt(a):
        return torch.nn.functional.conv2d(a[None], w2, padding=5, groups=3)[0]

    mx, my = filt(tx), filt(ty)
    sxx, syy, sxy = filt(tx * tx) - mx * mx, filt(ty * ty) - my * my, filt(tx * ty) - mx * my
    smap = (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    tl = (1 - lam) * (tx - ty).abs().mean() + lam * (1 - smap.mean())
    tl.backward()
    assert loss == pytest.approx(tl.item(), rel=1e-12)
    assert ssim == pytest.approx(smap.mean().item(), rel=1e-12)
    np.testing.assert_allclose(g, tx.grad.numpy(), rtol=1e-9, atol=1e-15)
