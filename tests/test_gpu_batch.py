"""GPU tests of the multi-view batch path (igs_render_batch): every view of a
batch is bit-identical to rendering it alone (which the oracle parity tests
pin), eagerly and through a captured CUDA graph, across tile sizes, staging
depths, several groups and new poses; overflow is reported."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_14244_gb300 import igs, scenes
from paper_2403_14244_gb300.batch import BatchRenderer, autotune, pack_groups
from tests import _gpu

pytestmark = pytest.mark.gpu


def _cams(seed=3):
    sizes = [(640, 360), (1280, 720), (333, 217), (800, 600), (96, 64)]
    rng = np.random.default_rng(seed)
    cams = []
    for w, h in sizes:
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        cams.append(scenes.pinhole(u * rng.uniform(3, 5), w, h, 0.866 * w))
    return cams


def _single(scene_np, cam, tile, footprint=0):
    return _gpu.run_forward(scene_np, cam, tile=tile, footprint=footprint)[3]


@pytest.mark.parametrize("tile,bb,footprint", [(16, 0, 0), (16, 64, 0), (8, 32, 0), (32, 512, 0), (32, 64, 0), (16, 128, 1),
                                               (8, 64, 1)])
def test_batch_bit_identical_to_single_renders(tile, bb, footprint):
    sc = scenes.uniform_scene(200_000, 41)
    scene = _gpu.to_device(sc)
    cams = _cams()
    br = BatchRenderer(scene, cams, tile=tile, blend_batch=bb, footprint=footprint)
    br.render()
    torch.cuda.synchronize()
    br.check()
    for v, cam in enumerate(cams):
        got = br.image(v).cpu().numpy().astype(np.float64)
        np.testing.assert_array_equal(got, _single(sc, cam, tile, footprint), err_msg=f"view {v}")


def test_batch_graph_replay_and_new_poses():
    sc = scenes.clustered_scene(150_000, 42, sh_degree=3)
    scene = _gpu.to_device(sc)
    cams = _cams(5)
    br = BatchRenderer(scene, cams, tile=16, sh_degree=3)
    br.capture()
    br.replay()
    torch.cuda.synchronize()
    for v, cam in enumerate(cams):
        np.testing.assert_array_equal(br.image(v).cpu().numpy().astype(np.float64), _single(sc, cam, 16))
    # new poses at the same image sizes: replay the same graph
    new = []
    for c in cams:
        R = c.R.astype(np.float64)
        ang = 0.1
        Ry = np.array([[np.cos(ang), 0, np.sin(ang)], [0, 1, 0], [-np.sin(ang), 0, np.cos(ang)]])
        c2 = scenes.Camera(R=(R @ Ry).astype(np.float32), t=c.t, fx=c.fx, fy=c.fy, cx=c.cx, cy=c.cy,
                           width=c.width, height=c.height)
        new.append(c2)
    br.set_poses(new)
    br.replay()
    torch.cuda.synchronize()
    br.check()
    for v, cam in enumerate(new):
        np.testing.assert_array_equal(br.image(v).cpu().numpy().astype(np.float64), _single(sc, cam, 16))


def test_batch_several_groups():
    sc = scenes.uniform_scene(120_000, 43)
    scene = _gpu.to_device(sc)
    cams = _cams(7)
    br = BatchRenderer(scene, cams, tile=16, entry_budget=1_500_000)
    assert len(br.groups) > 1
    br.capture()
    br.replay()
    torch.cuda.synchronize()
    for v, cam in enumerate(cams):
        np.testing.assert_array_equal(br.image(v).cpu().numpy().astype(np.float64), _single(sc, cam, 16))


def test_batch_view_matches_oracle():
    sc = scenes.uniform_scene(20_000, 44)
    scene = _gpu.to_device(sc)
    cams = _cams(9)[2:4]
    br = BatchRenderer(scene, cams, tile=16)
    br.render()
    torch.cuda.synchronize()
    for v, cam in enumerate(cams):
        ref = oracle.render(sc, cam, mode=1, flag_margin=2e-5)
        _gpu.compare_images(br.image(v).cpu().numpy().astype(np.float64), ref["img"], ref["flag"])


def test_batch_capacity_overflow_reported():
    sc = scenes.uniform_scene(50_000, 45)
    scene = _gpu.to_device(sc)
    cams = [igs.camera(c) for c in _cams(11)[:2]]
    o = igs.opts(tile=16)
    b = igs.Batch(scene.n, cams, o, capacity=5000)
    b.set_views()
    b.images.fill_(-1.0)
    b.render(scene)
    st, info = b.status()
    assert st == igs.ERR_CAPACITY and info[3] > 5000
    assert torch.all(b.images == -1.0)


def test_batch_empty_and_all_culled_scenes_give_the_background():
    """An empty scene, and one whose Gaussians are all culled (opacity below
    1/255), render the background in every view, as a single render does."""
    cams = _cams(15)[:3]
    bg = (0.25, 0.5, 1.0)
    for sc in (scenes.Scene(means_sigma=np.zeros((0, 4), np.float32), opacity=np.zeros(0, np.float32),
                            color=np.zeros((0, 3), np.float32), sh_degree=-1, log_params=False),
               scenes.uniform_scene(1000, 47)):
        if sc.n:
            sc.opacity[:] = np.float32(0.001)             # can never reach alpha_min: culled
        scene = _gpu.to_device(sc)
        br = BatchRenderer(scene, cams, tile=16, bg=bg)
        br.render()
        torch.cuda.synchronize()
        br.check()
        for v, cam in enumerate(cams):
            got = br.image(v).cpu().numpy()
            np.testing.assert_array_equal(got, np.broadcast_to(np.array(bg, np.float32)[:, None, None], got.shape))


def test_pack_groups():
    assert pack_groups([5, 5, 5, 5], 10) == [[0, 1], [2, 3]]
    assert pack_groups([20, 1], 10) == [[0], [1]]


def test_autotune_picks_and_caches(tmp_path):
    sc = scenes.uniform_scene(60_000, 46)
    scene = _gpu.to_device(sc)
    cams = _cams(13)[:3]
    path = str(tmp_path / "tune.json")
    best, timings = autotune(scene, cams, candidates=[(16, 256), (8, 64)], reps=2, cache_path=path)
    assert best in ((16, 256), (8, 64)) and len(timings) == 2
    best2, _ = autotune(scene, cams, candidates=[(32, 1024)], reps=2, cache_path=path)
    assert best2 == best                                  # served from the cache
