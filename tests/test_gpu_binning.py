"""GPU parity of the key path: projection, culling, tile rectangles, the
front-to-back (tile, depth) order and per-tile ranges, bit-exact against the
oracle's canonical FP32 key path and stable sort."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_14244_gb300 import igs, scenes
from tests import _gpu
from tests._tiny import scene_from, small_camera

pytestmark = pytest.mark.gpu


def _check_bitexact(sc, cam, tile, footprint=0):
    r, f, scene, img = _gpu.run_forward(sc, cam, tile=tile, footprint=footprint)
    p = oracle.project(sc.means_sigma, sc.opacity, cam, tile, footprint)
    count = f.count().cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(count, p["count"].astype(np.uint32))
    kept = p["count"] > 0
    rec = f.rec().cpu().numpy()
    np.testing.assert_array_equal(rec[kept, 0].view(np.uint32), p["u"][kept].view(np.uint32))
    np.testing.assert_array_equal(rec[kept, 1].view(np.uint32), p["v"][kept].view(np.uint32))
    # w2 = log2(e) / (2 s^2) rounded from the oracle's s; o as given; pmax a
    # bound on the exponent of every pixel whose alpha reaches alpha_min
    s_ = p["s"][kept]
    w2 = np.float32(np.float32(0.5) * np.float32(np.log2(np.e))) / (s_ * s_)
    np.testing.assert_array_equal(rec[kept, 2].view(np.uint32), w2.view(np.uint32))
    if not sc.log_params:
        np.testing.assert_array_equal(rec[kept, 7].view(np.uint32), sc.opacity[kept].view(np.uint32))
    bound = np.log2(rec[kept, 7].astype(np.float64) / np.float64(np.float32(1.0 / 255.0)))
    assert np.all(rec[kept, 3] >= bound + 2.0 ** -11) and np.all(rec[kept, 3] <= bound + 2.0 ** -9)
    dk = f.depth_key().cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(dk[kept], p["depth"][kept].view(np.uint32))
    assert np.all(dk[~kept] == 0xFFFFFFFF)
    rect = f.rect().cpu().numpy().view(np.uint32)
    x0, y0, x1, y1 = rect[:, 0] & 0xFFFF, rect[:, 0] >> 16, rect[:, 1] & 0xFFFF, rect[:, 1] >> 16
    np.testing.assert_array_equal(np.stack([x0, y0, x1, y1], 1)[kept], p["rect"][kept])
    keys, vals, ranges, info = _gpu.frame_keys(f)
    k_ref, v_ref, r_ref = oracle.keys(p, cam, tile)
    assert info[0] == len(k_ref)
    assert info[1] == int(kept.sum())
    np.testing.assert_array_equal(keys, k_ref)
    np.testing.assert_array_equal(vals, v_ref)
    np.testing.assert_array_equal(ranges, r_ref)
    return len(k_ref)


@pytest.mark.parametrize("footprint", [0, 1])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_keys_forward_4k(tile, footprint):
    sc, cam = scenes.workload_forward_4k()
    m = _check_bitexact(sc, cam, tile, footprint)
    assert m > 4096


@pytest.mark.parametrize("footprint", [0, 1])
def test_keys_ragged_large(footprint):
    # 1297 x 840 (ragged edge tiles), 300k Gaussians: many sort blocks, partial last block
    sc = scenes.uniform_scene(300_000, 7)
    cam = scenes.ring_cameras(16, 4.0, 1297, 840, 1100.0, cx=648.5, cy=420.0)[3]
    assert _check_bitexact(sc, cam, 16, footprint) > 1_000_000


def test_keys_clustered_sh_1080p_full():
    sc, cam, _ = scenes.workload_fwd_bwd_1m()
    _check_bitexact(sc, cam, 16)


@pytest.mark.parametrize("footprint", [0, 1])
@pytest.mark.parametrize("tile", [8, 32])
def test_keys_clustered_tiles(tile, footprint):
    sc = scenes.clustered_scene(200_000, 12)
    cam = scenes.pinhole((0.3, -0.1, -3.5), 1920, 1080, 1100.0)
    _check_bitexact(sc, cam, tile, footprint)


@pytest.mark.parametrize("footprint", [0, 1])
@pytest.mark.parametrize("width,route", [(16384, "counting"), (16392, "radix")])
def test_keys_both_routes(width, route, footprint):
    # 2048 tiles across at tile 8 is the widest frame the counting sort takes;
    # one more tile column sends the entries through duplication + radix passes
    sc = scenes.clustered_scene(200_000, 14)
    cam = scenes.pinhole((0.0, 0.0, -3.0), width, 40, 2000.0)
    f = igs.Frame(sc.n, 1 << 16, igs.camera(cam), igs.opts(tile=8))
    assert (f.struct.sort_chunks > 0) == (route == "counting")
    assert _check_bitexact(sc, cam, 8, footprint) > 10_000


@pytest.mark.parametrize("n", [1, 255, 257, 5000])
def test_keys_counting_sort_few_gaussians(n):
    # fewer Gaussians than one chunk, one chunk plus one, a handful of chunks
    sc = scenes.uniform_scene(n, 13)
    cam = scenes.pinhole((0.0, 0.0, -2.5), 640, 360, 600.0)
    _check_bitexact(sc, cam, 16)


def test_keys_edge_cases():
    cam = small_camera(40, 24, 64.0)
    # one Gaussian covering every tile, one off screen, one behind the near plane,
    # one with opacity below 1/255, one exactly on a tile corner, duplicates of depth
    means = [[0, 0, 0], [30, 0, 0], [0, 0, -3.999], [0.1, 0.1, 0], [0.5, 0.25, 0], [0.5, 0.25, 0]]
    sigma = [5.0, 0.1, 0.1, 0.1, 0.05, 0.05]
    opac = [0.5, 0.5, 0.5, 0.003, 0.7, 0.7]
    col = np.random.default_rng(0).uniform(size=(6, 3))
    sc = scene_from(means, sigma, opac, col)
    for tile in (8, 16, 32):
        for footprint in (0, 1):
            _check_bitexact(sc, cam, tile, footprint)


def test_empty_and_all_culled():
    cam = small_camera(48, 32, 64.0)
    sc = scene_from(np.zeros((0, 3)), [], [], np.zeros((0, 3)))
    r, f, scene, img = _gpu.run_forward(sc, cam)
    assert np.all(img == 0.0)
    sc = scene_from([[0, 0, -10.0]] * 5, [0.1] * 5, [0.5] * 5, np.ones((5, 3)))   # all behind the camera
    r, f, scene, img = _gpu.run_forward(sc, cam, bg=(0.25, 0.5, 1.0))
    np.testing.assert_array_equal(img, np.broadcast_to(np.array([0.25, 0.5, 1.0])[:, None, None], img.shape))
    st, info = igs.frame_status(f)
    assert st == igs.OK and info[0] == 0 and info[1] == 0


def test_capacity_overflow_is_reported():
    sc, cam = scenes.workload_forward_4k()
    scene = _gpu.to_device(sc)
    o = igs.opts(tile=16)
    c = igs.camera(cam)
    f = igs.Frame(scene.n, 1000, c, o)
    img = torch.full((3, 256, 256), -1.0, device="cuda")
    igs.project(scene, c, o, f)
    igs.bin_sort(f, o)
    igs.render_fwd(f, o, img)
    st, info = igs.frame_status(f)
    p = oracle.project(sc.means_sigma, sc.opacity, cam, 16)
    assert st == igs.ERR_CAPACITY
    assert info[3] == int(p["count"].sum())
    assert torch.all(img == -1.0)                      # outputs left untouched


def test_invalid_arguments_rejected():
    sc, cam = scenes.workload_forward_4k()
    o = igs.opts(tile=12)
    with pytest.raises(igs.IgsError) as e:
        igs.Frame(sc.n, 1 << 16, igs.camera(cam), o)
    assert e.value.status == igs.ERR_INVALID_ARG
    cam.fy = cam.fx * 1.01
    with pytest.raises(igs.IgsError):
        igs.Frame(sc.n, 1 << 16, igs.camera(cam), igs.opts(tile=16))


def _depth_scene(z, seed, W=640, H=480, f=500.0):
    """Gaussians at depths z (exactly: the camera sits at the origin with R = I),
    spread over the image; a tenth of them behind the camera (culled)."""
    rng = np.random.default_rng(seed)
    n = len(z)
    z = np.asarray(z, np.float32).copy()
    z[rng.random(n) < 0.1] *= np.float32(-1.0)
    u, v = rng.uniform(0, W, n), rng.uniform(0, H, n)
    means = np.stack([(u - W / 2) * np.abs(z) / f, (v - H / 2) * np.abs(z) / f, np.zeros(n)], 1)
    sc = scene_from(means, rng.uniform(0.005, 0.02, n), rng.uniform(0.2, 0.9, n), rng.uniform(0, 1, (n, 3)))
    sc.means_sigma[:, 2] = z                       # the depth bits exactly as drawn
    cam = scenes.Camera(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=f, fy=f, cx=W / 2, cy=H / 2,
                        width=W, height=H)
    return sc, cam


@pytest.mark.parametrize("case,skip", [("one_top_byte", 1), ("three_top_bytes", 0), ("low24_all_ones", 0)])
def test_depth_order_top_pass_skip(case, skip):
    """The depth sort skips its top-byte pass exactly when every kept key shares
    its top byte and none has its low 24 bits all ones; either way the order is
    the stable argsort of the depth keys (culled keys last, by index), and the
    keys and ranges stay bit-exact."""
    rng = np.random.default_rng(91)
    n = 60_001                                     # several radix blocks and a ragged last one
    if case == "three_top_bytes":
        z = rng.uniform(1.2, 12.0, n)              # exponents 127..130: top bytes 0x3F, 0x40, 0x41
    else:
        z = rng.uniform(2.3, 5.7, n)               # exponents 128, 129: top byte 0x40
    z = z.astype(np.float32)
    z[::7] = z[1::7][: z[::7].shape[0]]            # equal depths: ties by index
    sc, cam = _depth_scene(z, 92)
    if case == "low24_all_ones":                   # at the image centre, 7.9999995: kept, low 24 bits all ones
        sc.means_sigma[12345, :3] = np.array([0.0, 0.0, np.uint32(0x40FFFFFF).view(np.float32)], np.float32)
    _check_bitexact(sc, cam, 16)
    r, f, scene, img = _gpu.run_forward(sc, cam, tile=16)
    info = f.info().cpu().numpy().view(np.uint32)
    assert int(info[7]) == skip
    dk = f.depth_key().cpu().numpy().view(np.uint32)
    want = np.argsort(dk, kind="stable").astype(np.uint32)
    np.testing.assert_array_equal(f.order().cpu().numpy().view(np.uint32), want)
    assert (dk == 0xFFFFFFFF).sum() > 1000
