"""Pins of the oracle's FP32 key path: projection values, tile rectangles,
(tile, depth) keys, their stable order and the per-tile ranges.

The rectangle is pinned by what it must be (the smallest set of tiles that
holds every pixel a Gaussian can reach with alpha >= 1/255, up to the
footprint radius, itself pinned against FP64 logarithms), the order by numpy's
stable sort, the ranges by searchsorted.
"""

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


@pytest.mark.parametrize("footprint", [0, 1])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_rect_is_minimal_cover(tile, footprint):
    sc, cam = random_small(400, 3, w=70, h=50, spread=1.2)
    p = oracle.project(sc.means_sigma, sc.opacity, cam, tile, footprint)
    tx_n, ty_n = -(-cam.width // tile), -(-cam.height // tile)
    kept = p["count"] > 0
    assert kept.sum() > 100
    for i in np.nonzero(kept)[0]:
        u, v, r = float(p["u"][i]), float(p["v"][i]), float(p["r"][i])
        x0, y0, x1, y1 = p["rect"][i]
        assert 0 <= x0 <= x1 < tx_n and 0 <= y0 <= y1 < ty_n
        if footprint:
            xa, xb = oracle.row_span(p["u"][i], p["v"][i], p["r"][i], np.arange(y0, y1 + 1), x0, x1, tile)
            assert p["count"][i] == np.maximum(xb - xa + 1, 0).sum()
        else:
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


@pytest.mark.parametrize("footprint", [0, 1])
def test_rect_holds_every_reachable_pixel(footprint):
    """Every pixel where a Gaussian has alpha >= 1/255 (FP64 render of the
    Gaussian alone) lies in a tile it touches; off-grid ones never reach one."""
    sc, cam = random_small(60, 8, w=48, h=40, spread=1.0, smin=0.05, smax=0.3)
    for tile in (8, 16):
        p = oracle.project(sc.means_sigma, sc.opacity, cam, tile, footprint)
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
            # and in the touched tiles of its row
            xa, xb = oracle.row_span(np.full(len(ys), p["u"][i]), np.full(len(ys), p["v"][i]),
                                     np.full(len(ys), p["r"][i]), ys // tile, x0, x1, tile)
            assert np.all((xs // tile >= xa) & (xs // tile <= xb))


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_row_spans_are_the_tiles_the_disc_meets(tile):
    """Within the rectangle, a tile is in its row's span exactly when the disc
    of radius r meets the tile's square (FP64 distance from the centre to the
    square), up to a 1e-5 relative band for the FP32 roundings."""
    sc, cam = random_small(300, 21, w=150, h=110, spread=1.1, smin=0.05, smax=0.4)
    p = oracle.project(sc.means_sigma, sc.opacity, cam, tile, footprint=1)
    kept = np.nonzero(p["count"] > 0)[0]
    assert len(kept) > 100
    inside = outside = 0
    for i in kept:
        u, v, r = (float(p[k][i]) for k in ("u", "v", "r"))
        x0, y0, x1, y1 = p["rect"][i]
        rows = np.arange(y0, y1 + 1)
        xa, xb = oracle.row_span(np.full(len(rows), p["u"][i]), np.full(len(rows), p["v"][i]),
                                 np.full(len(rows), p["r"][i]), rows, x0, x1, tile)
        total = 0
        for ty, a, b in zip(rows, xa, xb):
            tx = np.arange(x0, x1 + 1)
            dx = np.maximum(0.0, np.maximum(tx * tile - u, u - (tx + 1) * tile))
            dy = max(0.0, ty * tile - v, v - (ty + 1) * tile)
            d = np.hypot(dx, dy)
            span = (tx >= a) & (tx <= b)
            assert np.all(span[d < r * (1 - 1e-5)]), (i, ty)
            assert not np.any(span[d > r * (1 + 1e-5)]), (i, ty)
            inside += int(span.sum())
            outside += int((~span).sum())
            total += int(span.sum())
        assert total == p["count"][i]
    assert outside > 0                      # the corner tiles of larger discs are left out


def test_radius_bounds_the_cutoff_tightly():
    """Eq. 2's support per particle: beyond r, alpha = o exp(-d^2/(2 s^2)) falls
    below 1/255 with room to spare (r^2 >= 2 s^2 (ln(255 o) + 2^-9), which holds
    the blend's own exponent slack of 2^-10 ln 2), and r is no more than 0.1 %
    above that bound. FP64 logarithms against the oracle's FP32 series."""
    o = np.concatenate([np.float32(1 / 255) * (1 + np.arange(64, dtype=np.float32) / 8),
                        np.linspace(0.01, 1.0, 4001, dtype=np.float32), np.float32([2.0, 7.5, 100.0])])
    o = o[o >= np.float32(1 / 255)].astype(np.float32)
    for s in (np.float32(0.37), np.float32(1.0), np.float32(23.5)):
        r = oracle.radius(np.full(o.shape, s, np.float32), o).astype(np.float64)
        ln = np.log(255.0 * o.astype(np.float64))
        need = float(s) * np.sqrt(2 * (ln + 2.0 ** -9))
        assert np.all(r >= need * (1 - 1e-6))
        assert np.all(r <= need * (1 + 1e-3))
        # alpha at the radius: below the cutoff by more than the blend's exponent slack
        alpha_r = o.astype(np.float64) * np.exp(-(r / float(s)) ** 2 / 2)
        assert np.all(alpha_r * 2 ** (2.0 ** -10) < 1 / 255)
    # the bound follows the opacity: a faint Gaussian reaches less far
    r1 = oracle.radius([1.0, 1.0], [1.0, 0.05])
    assert r1[1] < 0.7 * r1[0]


@pytest.mark.parametrize("footprint", [0, 1])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_keys_match_library_stable_sort(tile, footprint):
    sc, cam = random_small(500, 4, w=90, h=60, spread=1.0)
    p = oracle.project(sc.means_sigma, sc.opacity, cam, tile, footprint)
    k, v, r = oracle.keys(p, cam, tile)
    tx_n = -(-cam.width // tile)
    gen_k, gen_v = [], []
    for i in range(sc.n):                                     # generation order: index, row-major tiles
        if p["count"][i] == 0:
            continue
        x0, y0, x1, y1 = p["rect"][i]
        zb = int(np.float32(p["depth"][i]).view(np.uint32))
        for ty in range(y0, y1 + 1):
            xa, xb = oracle.row_span(p["u"][i], p["v"][i], p["r"][i], ty, x0, x1, tile) if footprint else ([x0], [x1])
            for tx in range(int(xa[0]), int(xb[0]) + 1):
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
