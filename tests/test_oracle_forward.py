"""Pins of the oracle's forward compositing (Eq. 4 with the kernel of Eq. 8).

Each test fixes the oracle to something other than itself: closed forms of
one- and two-Gaussian images, the explicit-product form of Eq. 4 evaluated by
brute force, and invariants the method must satisfy.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2403_14244_gb300 import scenes
from tests._tiny import random_small, scene_from, small_camera

A_MIN = np.float32(1.0 / 255.0)


def test_one_gaussian_closed_form():
    # camera at (0,0,-4): z_c = 4; f = 64 -> s = 64 sigma / 4 = 2 px for sigma = 1/8;
    # the centre lands on (u, v) = (8, 8), i.e. on a pixel corner.
    cam = small_camera(16, 16, 64.0)
    rgb = (1.0, 0.5, 0.25)
    sc = scene_from([0, 0, 0], [0.125], [0.5], [rgb])
    out = oracle.render(sc, cam, mode=0)
    img = out["img"]
    for py in range(16):
        for px in range(16):
            d2 = (px + 0.5 - 8.0) ** 2 + (py + 0.5 - 8.0) ** 2
            a = min(0.99, 0.5 * math.exp(-d2 / (2 * 2.0 ** 2)))
            if a < float(A_MIN):
                a = 0.0
            for ch in range(3):
                assert img[ch, py, px] == pytest.approx(rgb[ch] * a, abs=1e-12)
            assert out["T"][py, px] == pytest.approx(1.0 - a, abs=1e-12)
    # a hand-checked value: pixel (7,7) is sqrt(0.5) from the centre -> a = 0.5 e^{-1/16}
    assert img[0, 7, 7] == pytest.approx(0.46970653140673793, abs=1e-12)
    # pixel (15, 7): d^2 = 56.5, a = 0.5 e^{-7.0625} = 4.28e-4 < 1/255 -> skipped
    assert img[0, 7, 15] == 0.0 and out["nb"][7, 15] == 0


def test_one_gaussian_alpha_clamp():
    cam = small_camera(16, 16, 64.0, cx=8.5, cy=8.5)       # centre on pixel (8,8)'s centre
    sc = scene_from([0, 0, 0], [0.125], [1.0], [(1, 1, 1)])
    out = oracle.render(sc, cam, mode=0)
    a_max = float(np.float32(0.99))                          # thresholds are FP32 constants
    assert out["img"][0, 8, 8] == pytest.approx(a_max, abs=1e-15)   # min(0.99, 1 * 1)
    assert out["T"][8, 8] == pytest.approx(1.0 - a_max, abs=1e-15)


def test_two_gaussians_order():
    # same screen position, different depths: C = c1 a1 + c2 a2 (1 - a1), front first
    cam = small_camera(16, 16, 64.0, cx=8.5, cy=8.5)
    front, back = (1.0, 0.0, 0.0), (0.0, 0.0, 1.0)
    # back Gaussian twice as far: z = 8 -> put it at world z = 4 with sigma doubled (same s)
    sc = scene_from([[0, 0, 0], [0, 0, 4]], [0.125, 0.25], [0.6, 0.7], [front, back])
    out = oracle.render(sc, cam, mode=0)
    a1, a2 = float(np.float32(0.6)), float(np.float32(0.7))   # inputs are stored in FP32
    assert out["img"][0, 8, 8] == pytest.approx(a1, abs=1e-12)
    assert out["img"][2, 8, 8] == pytest.approx(a2 * (1 - a1), abs=1e-12)
    assert out["T"][8, 8] == pytest.approx((1 - a1) * (1 - a2), abs=1e-12)
    assert out["last"][8, 8] == 1
    # listing order in the input does not matter, depth does
    sc2 = scene_from([[0, 0, 4], [0, 0, 0]], [0.25, 0.125], [0.7, 0.6], [back, front])
    out2 = oracle.render(sc2, cam, mode=0)
    np.testing.assert_array_equal(out["img"], out2["img"])


def test_transmittance_stop_rule():
    # five opaque discs stacked front to back, a = 0.9 each (o = 0.9, centred):
    # T: 1 -> 0.1 -> 0.01 -> 1e-3 -> 1e-4 (not < 1e-4? 1e-4*(1 +- eps)) -> stop
    cam = small_camera(16, 16, 64.0, cx=8.5, cy=8.5)
    zs = [0.0, 1.0, 2.0, 3.0, 4.0, 5.0]
    cols = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, 0, 1)]
    sig = [0.125 * (4 + z) / 4 for z in zs]                  # same s = 2 px at every depth
    sc = scene_from([[0, 0, z] for z in zs], sig, [0.9] * 6, cols)
    out = oracle.render(sc, cam, mode=0)
    # Explicit: T_k after k entries is 0.1^k; entry 4 would give 1e-4 * 0.1 = 1e-5 < 1e-4 -> stop
    # so entries 0..3 are blended and T_final = 0.1^4 = 1e-4 (T' of entry 3 = 1e-4 is not < 1e-4,
    # up to rounding; the flag records how close it is).
    nb = out["nb"][8, 8]
    assert nb in (3, 4)
    T = out["T"][8, 8]
    assert T >= 1e-4 * (1 - 1e-9)
    # every blended entry contributes 0.9 * 0.1^k of its colour
    expect = np.zeros(3)
    for k in range(nb):
        a = float(np.float32(0.9))
        expect += np.array(cols[k]) * a * (1 - a) ** k
    np.testing.assert_allclose(out["img"][:, 8, 8], expect, atol=1e-12)


def _explicit_product(sc, cam, bg=(0, 0, 0)):
    """Eq. 4 as an explicit sum of products (not the running-T recursion),
    over the Gaussians the cutoff and stop rules keep, per pixel, by brute force.
    Projection done here in float64 from the FP32 inputs."""
    ms = sc.means_sigma.astype(np.float64)
    R, t = cam.R.astype(np.float64), cam.t.astype(np.float64)
    xc = ms[:, :3] @ R.T + t
    z = xc[:, 2]
    u = cam.fx * xc[:, 0] / z + cam.cx
    v = cam.fy * xc[:, 1] / z + cam.cy
    s = cam.fx * ms[:, 3] / z
    o = sc.opacity.astype(np.float64)
    col = sc.color.astype(np.float64)
    zf = (ms[:, :3].astype(np.float32) @ cam.R.T.astype(np.float32) + cam.t).astype(np.float32)[:, 2]
    order = np.lexsort((np.arange(sc.n), z))                # depth, then index
    H, W = cam.height, cam.width
    img = np.zeros((3, H, W))
    for py in range(H):
        for px in range(W):
            alphas, cs = [], []
            for i in order:
                if not z[i] > cam.znear or o[i] < float(A_MIN):
                    continue
                d2 = (px + 0.5 - u[i]) ** 2 + (py + 0.5 - v[i]) ** 2
                a = min(0.99, o[i] * math.exp(-d2 / (2 * s[i] ** 2)))
                if a < float(A_MIN):
                    continue
                if np.prod([1 - x for x in alphas]) * (1 - a) < 1e-4:
                    break
                alphas.append(a)
                cs.append(col[i])
            c = np.zeros(3)
            for k in range(len(alphas)):
                c += cs[k] * alphas[k] * np.prod([1 - alphas[j] for j in range(k)])
            c += np.prod([1 - x for x in alphas]) * np.asarray(bg)
            img[:, py, px] = c
    del zf
    return img


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_explicit_product_form(seed):
    sc, cam = random_small(14, seed, w=18, h=14)
    got = oracle.render(sc, cam, mode=0, proj64=True, bg=(0.25, 0.5, 0.125))
    want = _explicit_product(sc, cam, bg=(0.25, 0.5, 0.125))
    # decisions within 1e-9 of a threshold could legitimately differ; none expected here
    assert got["flag"].sum() == 0
    np.testing.assert_allclose(got["img"], want, atol=1e-12, rtol=0)


@pytest.mark.parametrize("sh", [-1, 3])
def test_literal_equals_lists_bitwise(sh):
    sc, cam = random_small(300, 7, w=40, h=30, sh_degree=sh, spread=0.8)
    a = oracle.render(sc, cam, mode=0)
    b = oracle.render(sc, cam, mode=1)
    for k in ("img", "T", "nb", "last", "flag", "hash"):
        np.testing.assert_array_equal(a[k], b[k])


def test_invariants_forward_4k():
    sc, cam = scenes.workload_forward_4k()
    out = oracle.render(sc, cam, mode=1)
    img, T = out["img"], out["T"]
    assert np.all(T <= 1.0) and np.all(T >= 1e-4)           # stop keeps T >= t_min
    assert np.all(img >= 0.0)
    cmax = sc.color.max(axis=0).astype(np.float64)
    # bg = 0: each channel is a convex-like mix, bounded by (1 - T) * max colour
    assert np.all(img <= (1.0 - T)[None] * cmax[:, None, None] + 1e-12)
    assert np.all((out["nb"] == 0) == (out["last"] == -1))
    assert np.all((out["nb"] == 0) <= (T == 1.0))


def test_shuffle_invariance_bitwise():
    sc, cam = random_small(200, 11, w=32, h=24, sh_degree=3, spread=0.8)
    perm = np.random.default_rng(0).permutation(sc.n)
    sc2 = scenes.Scene(sc.means_sigma[perm].copy(), sc.opacity[perm].copy(), sc.color[perm].copy(), 3)
    a = oracle.render(sc, cam, mode=1)
    b = oracle.render(sc2, cam, mode=1)
    z = (sc.means_sigma[:, :3] @ cam.R.T + cam.t)[:, 2]
    assert len(np.unique(z)) == sc.n                          # distinct depths
    np.testing.assert_array_equal(a["img"], b["img"])
    np.testing.assert_array_equal(a["T"], b["T"])
    blended = a["last"] >= 0
    np.testing.assert_array_equal(perm[b["last"][blended]], a["last"][blended])


def test_rigid_motion_invariance():
    sc, cam = random_small(120, 5, w=32, h=24, sh_degree=3, spread=0.8)
    rng = np.random.default_rng(3)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    p = rng.normal(size=3)
    ms2 = sc.means_sigma.copy()
    ms2[:, :3] = (sc.means_sigma[:, :3].astype(np.float64) @ q.T + p).astype(np.float32)
    # SH coefficients live in world directions: rotate the direction argument instead by
    # using only the DC band for this check
    col = sc.color.reshape(sc.n, 16, 3).copy()
    col[:, 1:, :] = 0
    sc_a = scenes.Scene(sc.means_sigma, sc.opacity, col.reshape(sc.n, 48), 3)
    sc_b = scenes.Scene(ms2, sc.opacity, col.reshape(sc.n, 48), 3)
    R2 = (cam.R.astype(np.float64) @ q.T)
    t2 = cam.t.astype(np.float64) - R2 @ p
    cam2 = scenes.Camera(R=R2.astype(np.float32), t=t2.astype(np.float32), fx=cam.fx, fy=cam.fy, cx=cam.cx,
                         cy=cam.cy, width=cam.width, height=cam.height)
    a = oracle.render(sc_a, cam, mode=1, proj64=True, flag_margin=1e-4)
    b = oracle.render(sc_b, cam2, mode=1, proj64=True, flag_margin=1e-4)
    ok = (a["flag"] == 0) & (b["flag"] == 0)
    assert ok.mean() > 0.95
    np.testing.assert_allclose(a["img"][:, ok], b["img"][:, ok], atol=2e-5)


def test_background_uses_final_transmittance():
    sc, cam = random_small(40, 9, w=20, h=16)
    a = oracle.render(sc, cam, mode=1)
    b = oracle.render(sc, cam, mode=1, bg=(0.25, 0.5, 1.0))
    bg = np.array([0.25, 0.5, 1.0])[:, None, None]
    np.testing.assert_allclose(b["img"], a["img"] + a["T"][None] * bg, atol=1e-15)


def test_culling_rules():
    cam = small_camera(16, 16, 64.0, cx=8.5, cy=8.5)
    # behind the near plane (camera at z=-4), opacity below 1/255, far off screen
    sc = scene_from([[0, 0, -4.0 + 0.005], [0, 0, 0], [0, 0, 0], [50, 0, 0]],
                    [0.125, 0.125, 0.125, 0.125], [0.9, 0.9, 0.0039, 0.9],
                    [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)])
    out = oracle.render(sc, cam, mode=0)
    assert out["n_visible"] == 2                              # near-plane and o < 1/255 culled
    assert out["img"][2].max() == 0.0                         # o < 1/255 never blends
    assert out["img"][1, 8, 8] == pytest.approx(float(np.float32(0.9)), abs=1e-12)
