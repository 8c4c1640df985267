"""Pins of the oracle's FP32 key path: projection values, tile rectangles,
(tile, depth) keys, their stable order and the per-tile ranges.

The rectangle is pinned by what it must be (the smallest set of tiles that
holds every pixel a Gaussian can reach with alpha >= 1/255, up to the fixed
3.33 s radius), the order by numpy's stable sort, the ranges by searchsorted.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2403_14244_gb300 import scenes
from tests._tiny import random_small


def _proj64(sc, cam):
    ms = sc.means_sigma.astype(np.float64)
    xc = ms[:, :3] @ cam.R.astype(np.float64).T + cam.t.astype(np.float64)
    z = xc[:, 2]
    return (cam.fx * xc[:, 0] / z + cam.cx, cam.fy * xc[:, 1] / z + cam.cy, cam.fx * ms[:, 3] / z, z)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_projection_close_to_fp64(tile):
    sc, cam = scenes.workload_forward_4k()
    p = oracle.project(sc.means_sigma, sc.opacity, cam, tile)
    u, v, s, z = _proj64(sc, cam)
    # FP32 with a handful of single roundings: a few ulp of the magnitude
    np.testing.assert_allclose(p["u"], u, rtol=0, atol=4 * np.spacing(np.float32(256)))
    np.testing.assert_allclose(p["v"], v, rtol=0, atol=4 * np.spacing(np.float32(256)))
    np.testing.assert_allclose(p["s"], s, rtol=4e-7)
    np.testing.assert_allclose(p["depth"], z, rtol=4e-7)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_rect_is_minimal_cover(tile):
    sc, cam = random_small(400, 3, w=70, h=50, spread=1.2)
    p = oracle.project(sc.means_sigma, sc.opacity, cam, tile)
    tx_n, ty_n = -(-cam.width // tile), -(-cam.height // tile)
    kept = p["count"] > 0
    assert kept.sum() > 100
    for i in np.nonzero(kept)[0]:
        u, v, r = float(p["u"][i]), float(p["v"][i]), 3.33 * float(p["s"][i])
        x0, y0, x1, y1 = p["rect"][i]
        assert 0 <= x0 <= x1 < tx_n and 0 <= y0 <= y1 < ty_n
        assert p["count"][i] == (x1 - x0 + 1) * (y1 - y0 + 1)
        # the first and last tile of each axis hold the ends of [u-r, u+r] (resp. v), unless
        # the end lies off the grid and the rect is clamped; so the rect is the smallest
        # run of tiles covering the interval (allowing FP32 rounding of the ends)
        eps = 1e-4 * max(1.0, abs(u) + r, abs(v) + r)
        for lo_t, hi_t, c, n_t in ((x0, x1, u, tx_n), (y0, y1, v, ty_n)):
            if lo_t > 0:
                assert lo_t * tile <= c - r + eps and c - r < (lo_t + 1) * tile + eps
            else:
                assert c - r < tile + eps
            if hi_t < n_t - 1:
                assert hi_t * tile <= c + r + eps and c + r < (hi_t + 1) * tile + eps
            else:
                assert c + r >= hi_t * tile - eps


def test_rect_holds_every_reachable_pixel():
    """Every pixel where a Gaussian has alpha >= 1/255 (FP64 render of the
    Gaussian alone) lies in a tile of its rectangle; off-grid ones never reach one."""
    sc, cam = random_small(60, 8, w=48, h=40, spread=1.0, smin=0.05, smax=0.3)
    for tile in (8, 16):
        p = oracle.project(sc.means_sigma, sc.opacity, cam, tile)
        for i in range(sc.n):
            one = scenes.Scene(sc.means_sigma[i:i + 1].copy(), sc.opacity[i:i + 1].copy(),
                               sc.color[i:i + 1].copy(), -1)
            out = oracle.render(one, cam, mode=0)
            ys, xs = np.nonzero(out["nb"] > 0)
            if p["count"][i] == 0:
                assert len(xs) == 0
                continue
            x0, y0, x1, y1 = p["rect"][i]
            assert np.all((xs // tile >= x0) & (xs // tile <= x1))
            assert np.all((ys // tile >= y0) & (ys // tile <= y1))


def test_radius_constant_bounds_the_cutoff():
    # o exp(-K^2/2) < 1/255 for every o <= 1 with K = 3.33 (the footprint reading of Eq. 2)
    assert math.exp(-3.33 ** 2 / 2) < float(np.float32(1 / 255))


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_keys_match_library_stable_sort(tile):
    sc, cam = random_small(500, 4, w=90, h=60, spread=1.0)
    p = oracle.project(sc.means_sigma, sc.opacity, cam, tile)
    k, v, r = oracle.keys(p, cam, tile)
    tx_n = -(-cam.width // tile)
    gen_k, gen_v = [], []
    for i in range(sc.n):                                     # generation order: index, row-major tiles
        if p["count"][i] == 0:
            continue
        x0, y0, x1, y1 = p["rect"][i]
        zb = int(np.float32(p["depth"][i]).view(np.uint32))
        for ty in range(y0, y1 + 1):
            for tx in range(x0, x1 + 1):
                gen_k.append(((ty * tx_n + tx) << 32) | zb)
                gen_v.append(i)
    gen_k = np.array(gen_k, np.uint64)
    gen_v = np.array(gen_v, np.uint32)
    order = np.argsort(gen_k, kind="stable")
    np.testing.assert_array_equal(k, gen_k[order])
    np.testing.assert_array_equal(v, gen_v[order])
    tiles = (k >> np.uint64(32)).astype(np.int64)
    n_tiles = r.shape[0]
    lo = np.searchsorted(tiles, np.arange(n_tiles), side="left")
    hi = np.searchsorted(tiles, np.arange(n_tiles), side="right")
    empty = lo == hi
    np.testing.assert_array_equal(r[~empty, 0], lo[~empty])
    np.testing.assert_array_equal(r[~empty, 1], hi[~empty])
    assert np.all(r[empty] == 0)


def test_depth_key_orders_front_to_back():
    sc, cam = scenes.workload_forward_4k()
    p = oracle.project(sc.means_sigma, sc.opacity, cam, 16)
    k, v, r = oracle.keys(p, cam, 16)
    for t in range(r.shape[0]):
        a, b = r[t]
        d = p["depth"][v[a:b]]
        assert np.all(np.diff(d) >= 0)                        # positive floats: bits order = value order


def test_key_culling():
    sc, cam = random_small(50, 2, w=20, h=20)
    ms = sc.means_sigma.copy()
    op = sc.opacity.copy()
    ms[0, 3] = -1.0                                          # sigma <= 0
    ms[1, 0] = np.nan                                        # non-finite
    op[2] = np.float32(0.0039)                               # below 1/255
    ms[3, :3] = cam.center() + 0.001 * cam.R[2]              # just in front of the camera: z < znear
    ms[4, 0] = 1e3                                           # far off screen
    p = oracle.project(ms, op, cam, 16)
    assert np.all(p["count"][:5] == 0)


def test_tile_base_offsets_keys():
    sc, cam = random_small(80, 6, w=40, h=30)
    p = oracle.project(sc.means_sigma, sc.opacity, cam, 8)
    k0, v0, r0 = oracle.keys(p, cam, 8)
    k1, v1, r1 = oracle.keys(p, cam, 8, tile_base=1000)
    np.testing.assert_array_equal(v0, v1)
    np.testing.assert_array_equal(k1 - k0, np.full(k0.shape, 1000 << 32, np.uint64))
    np.testing.assert_array_equal(r0, r1)
