"""GPU tests of the render server (igs_serve_*): every result is identical
alone and in a concurrent mix, overflowing requests are re-queued with the
capacity they need, requests that can never fit are refused, and admission
never exceeds the pool."""
import numpy as np
import pytest
import torch

from paper_2403_14244_gb300 import igs, scenes
from tests import _gpu

pytestmark = pytest.mark.gpu

SIZES = [(854, 480), (1280, 720), (333, 217), (1920, 1080), (640, 360)]


def _requests(k, seed, n_scenes):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        w, h = SIZES[int(rng.integers(0, len(SIZES)))]
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        out.append((int(rng.integers(0, n_scenes)), scenes.pinhole(u * rng.uniform(3, 5), w, h, 0.866 * w)))
    return out


def _serve(srv, sids, reqs):
    outs = [torch.full((3, c.height, c.width), -1.0, device="cuda") for _, c in reqs]
    ids = [srv.submit(sids[s], c, o) for (s, c), o in zip(reqs, outs)]
    timings = []
    for i in ids:
        st, t = srv.poll(i, timeout_s=30.0)
        assert st == igs.OK, st
        timings.append(t)
    return outs, timings


@pytest.mark.parametrize("slots,group,tile", [(1, 1, 16), (4, 1, 16), (1, 8, 16), (4, 8, 32), (2, 4, 8)])
def test_results_identical_alone_and_in_the_mix(slots, group, tile):
    """Every image served in a concurrent mix, with or without grouping of a
    scene's waiting requests into one batched chain, equals the image of
    rendering that request alone, bit for bit. With grouping on, groups form
    once every (scene, size) has been seen (a second round of the same
    requests) and the requests of one group report its size."""
    scs = [scenes.uniform_scene(150_000, 51), scenes.clustered_scene(100_000, 52, sh_degree=3)]
    devs = [_gpu.to_device(s) for s in scs]
    srv = igs.Server(pool_bytes=3 << 30, slots=slots, tile=tile, group=group)
    sids = [srv.add_scene(d, sh_degree=s.sh_degree) for d, s in zip(devs, scs)]
    reqs = _requests(14, 53, len(scs))
    _serve(srv, sids, reqs)                 # first round: the capacity of every (scene, size) becomes known
    outs, timings = _serve(srv, sids, reqs)
    stats = srv.stats()
    srv.close()
    assert stats["pool_peak"] <= 3 << 30
    for (s, cam), o, t in zip(reqs, outs, timings):
        alone = _gpu.run_forward(scs[s], cam, tile=tile)[3]
        np.testing.assert_array_equal(o.cpu().numpy().astype(np.float64), alone)
        assert t["arrival_ns"] <= t["admit_ns"] <= t["start_ns"] <= t["done_ns"]
        assert 1 <= t["group"] <= group
    if group > 1:
        assert max(t["group"] for t in timings) > 1


def test_group_that_overflows_is_split_and_redone():
    """A group sized from small views of a scene, then asked for larger ones,
    overflows as a whole: its requests are redone one by one, each correct."""
    sc = scenes.uniform_scene(60_000, 57)
    sc.means_sigma[:, 3] *= 6.0
    dev = _gpu.to_device(sc)
    srv = igs.Server(pool_bytes=3 << 30, slots=1, tile=16, group=8)
    sid = srv.add_scene(dev)
    far = [scenes.pinhole((0.0, 0.0, -12.0 - 0.1 * k), 640, 360, 554.0) for k in range(6)]
    near = [scenes.pinhole((0.0, 0.0, -2.2 - 0.01 * k), 640, 360, 554.0) for k in range(6)]
    _serve(srv, [sid], [(0, c) for c in far])          # capacity hint from far (few entries per Gaussian)
    outs, timings = _serve(srv, [sid], [(0, c) for c in near])
    srv.close()
    assert any(t["retries"] >= 1 for t in timings)
    for cam, o in zip(near, outs):
        np.testing.assert_array_equal(o.cpu().numpy().astype(np.float64), _gpu.run_forward(sc, cam, tile=16)[3])


def test_overflow_is_requeued_with_the_needed_capacity():
    # large Gaussians: far more than 16 entries per Gaussian, so the first guess overflows
    sc = scenes.uniform_scene(20_000, 54)
    sc.means_sigma[:, 3] *= 12.0
    dev = _gpu.to_device(sc)
    srv = igs.Server(pool_bytes=2 << 30, slots=2, tile=8)
    sid = srv.add_scene(dev)
    cam = scenes.pinhole((0.0, 0.0, -4.0), 1280, 720, 1100.0)
    out = torch.full((3, 720, 1280), -1.0, device="cuda")
    st, t = srv.poll(srv.submit(sid, cam, out), timeout_s=30.0)
    srv.close()
    assert st == igs.OK and t["retries"] >= 1 and t["entries"] > 16 * sc.n
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), _gpu.run_forward(sc, cam, tile=8)[3])


def test_request_that_can_never_fit_is_refused():
    sc = scenes.uniform_scene(10_000, 55)
    srv = igs.Server(pool_bytes=1 << 20, slots=1)
    sid = srv.add_scene(_gpu.to_device(sc))
    cam = scenes.pinhole((0.0, 0.0, -4.0), 3840, 2160, 3325.0)
    with pytest.raises(igs.IgsError) as e:
        srv.submit(sid, cam, torch.empty((3, 2160, 3840), device="cuda"))
    srv.close()
    assert e.value.status == igs.ERR_CAPACITY


def test_poll_times_out_while_running():
    sc = scenes.uniform_scene(3_000_000, 56)
    srv = igs.Server(pool_bytes=8 << 30, slots=1)
    sid = srv.add_scene(_gpu.to_device(sc))
    cam = scenes.pinhole((0.0, 0.0, -4.0), 3840, 2160, 3325.0)
    out = torch.empty((3, 2160, 3840), device="cuda")
    rid = srv.submit(sid, cam, out)
    st, _ = srv.poll(rid, timeout_s=0.0)
    assert st == igs.ERR_NOT_READY
    st, t = srv.poll(rid, timeout_s=60.0)
    srv.close()
    assert st == igs.OK
