"""GPU parity of the forward blend (Eq. 4): images within 2e-4 of the FP64
oracle outside the pixels whose cutoff/stop decisions lie within the oracle's
margin; bit-identical across tile sizes; deterministic."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_14244_gb300 import igs, scenes
from tests import _gpu
from tests._tiny import random_small, scene_from

pytestmark = pytest.mark.gpu

MARGIN = 2e-5     # relative margin of the oracle's near-threshold flag


def _last_ids(f, vals_all, tile):
    """Gaussian id of each pixel's last blended entry on the GPU (-1 if none)."""
    nc = f.n_contrib().cpu().numpy().astype(np.int64)
    ranges = f.ranges().cpu().numpy().view(np.uint32).astype(np.int64)
    H, W = nc.shape
    ys, xs = np.mgrid[0:H, 0:W]
    t = (ys // tile) * f.tiles_x + (xs // tile)
    pos = ranges[t, 0] + nc - 1
    return np.where(nc > 0, vals_all[np.clip(pos, 0, None)], -1)


@pytest.mark.parametrize("footprint", [0, 1])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_forward_4k_matches_oracle(tile, footprint):
    sc, cam = scenes.workload_forward_4k()
    r, f, scene, img = _gpu.run_forward(sc, cam, tile=tile, footprint=footprint)
    ref = oracle.render(sc, cam, mode=1, flag_margin=MARGIN)
    _gpu.compare_images(img, ref["img"], ref["flag"])
    ok = ref["flag"] == 0
    T = f.T_final().cpu().numpy()
    np.testing.assert_allclose(T[ok], ref["T"][ok], atol=2e-4)
    keys, vals, ranges, info = _gpu.frame_keys(f)
    last = _last_ids(f, vals.astype(np.int64), tile)
    assert np.mean(last[ok] == ref["last"][ok]) == 1.0


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_footprints_give_the_same_image(tile):
    """Footprint 1 leaves out only tiles the disc does not meet, where no pixel
    reaches alpha_min: image and final transmittance are bit-identical, with
    fewer entries."""
    sc = scenes.clustered_scene(150_000, 23, sh_degree=3)
    cam = scenes.pinhole((0.4, -0.2, -3.2), 1280, 720, 1100.0)
    r0, f0, _, img0 = _gpu.run_forward(sc, cam, tile=tile, footprint=0)
    r1, f1, _, img1 = _gpu.run_forward(sc, cam, tile=tile, footprint=1)
    np.testing.assert_array_equal(img0, img1)
    np.testing.assert_array_equal(f0.T_final().cpu().numpy(), f1.T_final().cpu().numpy())
    assert igs.frame_status(f1)[1][0] < igs.frame_status(f0)[1][0]


def test_tile_sizes_bit_identical():
    sc = scenes.clustered_scene(100_000, 21)
    cam = scenes.pinhole((0.2, 0.1, -3.6), 640, 360, 560.0)
    imgs = [_gpu.run_forward(sc, cam, tile=t)[3] for t in (8, 16, 32)]
    np.testing.assert_array_equal(imgs[0], imgs[1])
    np.testing.assert_array_equal(imgs[0], imgs[2])


def test_deterministic():
    sc = scenes.clustered_scene(50_000, 22)
    cam = scenes.pinhole((0.0, 0.0, -4.0), 333, 217, 300.0)
    a = _gpu.run_forward(sc, cam)[3]
    b = _gpu.run_forward(sc, cam)[3]
    np.testing.assert_array_equal(a, b)


def test_sh3_log_params_small():
    sc, cam = random_small(400, 23, w=96, h=72, sh_degree=3, log_params=True, spread=0.8)
    r, f, scene, img = _gpu.run_forward(sc, cam, bg=(0.25, 0.5, 0.125))
    ref = oracle.render(sc, cam, mode=1, flag_margin=MARGIN, bg=(0.25, 0.5, 0.125))
    # log parameters: sigma, opacity activated in FP32 on the GPU vs FP64 in the oracle
    _gpu.compare_images(img, ref["img"], ref["flag"], atol=2e-4)


def test_forward_clustered_1080p_full():
    sc, cam, _ = scenes.workload_fwd_bwd_1m()
    r, f, scene, img = _gpu.run_forward(sc, cam)
    ref = oracle.render(sc, cam, mode=1, flag_margin=MARGIN)
    err = _gpu.compare_images(img, ref["img"], ref["flag"])
    assert err < 2e-4


def test_forward_train_view_full():
    sc, cams = scenes.workload_train_3m()
    cam = cams[5]
    r, f, scene, img = _gpu.run_forward(sc, cam)
    ref = oracle.render(sc, cam, mode=1, flag_margin=MARGIN)
    _gpu.compare_images(img, ref["img"], ref["flag"])


def test_autograd_function_forward_matches_renderer():
    from paper_2403_14244_gb300.render import Renderer, render
    sc, cam = scenes.workload_forward_4k()
    dev = _gpu.to_device(sc)
    r = Renderer(tile=16)
    img = render(dev.means_sigma, dev.opacity, dev.color, r, cam)
    ref = _gpu.run_forward(sc, cam)[3]
    np.testing.assert_array_equal(img.detach().cpu().numpy().astype(np.float64), ref)
    torch.cuda.synchronize()


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_alpha_threshold_decisions_exact(tile):
    """One small Gaussian per 16x16 block and one probe pixel at the edge of its
    disc, where alpha = alpha_min (1 + eps) with 1e-4 <= |eps| <= 2e-3 (in FP64
    from the FP32 u, v, s). The forward blends the probe exactly when eps > 0,
    and the backward sees it exactly then: no early skip (block of rows or
    per-pixel exponent bound) may drop a pair that reaches alpha_min."""
    rng = np.random.default_rng(77)
    W = H = 512
    f = 1000.0
    cam = scenes.Camera(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=f, fy=f,
                        cx=W / 2, cy=H / 2, width=W, height=H)
    amin = float(np.float32(1.0 / 255.0))
    n = (W // 16) * (H // 16)
    s_px = 1.5
    means, sig, opac, probes, eps_t = [], [], [], [], []
    for k in range(n):
        bi, bj = k % (W // 16), k // (W // 16)
        th = rng.uniform(0, 2 * np.pi)
        d = np.array([np.cos(th), np.sin(th)])
        o = rng.uniform(0.3, 0.9)
        eps = rng.uniform(2e-4, 1.5e-3) * (1 if k % 2 else -1)
        dist = s_px * np.sqrt(2 * np.log(o / (amin * (1 + eps))))
        P = np.floor(np.array([16 * bi + 8, 16 * bj + 8]) + 4.6 * d) + 0.5
        c = P - dist * d
        z = rng.uniform(3, 5)
        means.append([(c[0] - cam.cx) * z / f, (c[1] - cam.cy) * z / f, z])
        sig.append(s_px * z / f)
        opac.append(o)
        probes.append(P)
    sc = scene_from(means, sig, opac, rng.uniform(0.2, 1.0, size=(n, 3)))
    p = oracle.project(sc.means_sigma, sc.opacity, cam, tile)
    probes = np.array(probes)
    d2 = (probes[:, 0] - p["u"].astype(np.float64)) ** 2 + (probes[:, 1] - p["v"].astype(np.float64)) ** 2
    s64 = p["s"].astype(np.float64)
    eps_a = sc.opacity.astype(np.float64) * np.exp(-d2 / (2 * s64 * s64)) / amin - 1.0
    sel = (np.abs(eps_a) >= 1e-4) & (np.abs(eps_a) <= 2e-3)
    assert sel.sum() > 0.9 * n and (eps_a[sel] > 0).sum() > 0.4 * n
    r, fr, scene, img = _gpu.run_forward(sc, cam, tile=tile)
    px, py = probes[:, 0].astype(np.int64), probes[:, 1].astype(np.int64)
    nc = fr.n_contrib().cpu().numpy()[py, px]
    np.testing.assert_array_equal((nc > 0)[sel], (eps_a > 0)[sel])
    dimg = torch.zeros((3, H, W), device="cuda")
    dimg[:, torch.from_numpy(py).cuda(), torch.from_numpy(px).cuda()] = 1.0
    _, _, d_col = r.run_backward(scene, cam, fr, dimg)
    g = d_col.abs().sum(1).cpu().numpy()
    np.testing.assert_array_equal((g > 0)[sel], (eps_a > 0)[sel])


def test_frame_stats_match_the_oracle():
    """Per-frame counters (kept Gaussians, entries, per-tile list lengths)
    against the oracle's projection and keys; the reached list positions per
    pixel bounded by the tile lists."""
    sc, cam = scenes.workload_forward_4k()
    r, f, scene, img = _gpu.run_forward(sc, cam, tile=16)
    st = igs.frame_stats(f)
    keys, vals, ranges = oracle.keys(oracle.project(sc.means_sigma, sc.opacity, cam, 16), cam, 16)
    per_tile = ranges[:, 1].astype(np.int64) - ranges[:, 0].astype(np.int64)
    assert st["entries"] == len(keys) and st["entries_per_tile_max"] == per_tile.max()
    assert st["entries_per_tile_mean"] == pytest.approx(per_tile.mean())
    assert st["empty_tiles"] == pytest.approx(float((per_tile == 0).mean()))
    assert st["kept"] == int((oracle.project(sc.means_sigma, sc.opacity, cam, 16)["count"] > 0).sum())
    # a pixel's walk reaches at most its tile's list
    assert 0.0 < st["contrib_per_pixel_mean"] <= st["contrib_per_pixel_max"] <= per_tile.max()
    nc = f.n_contrib().cpu().numpy().astype(np.int64)
    assert st["contrib_per_pixel_mean"] == pytest.approx(nc.mean())
