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


@pytest.mark.parametrize("slots", [1, 4])
def test_results_identical_alone_and_in_the_mix(slots):
    scs = [scenes.uniform_scene(150_000, 51), scenes.clustered_scene(100_000, 52, sh_degree=3)]
    devs = [_gpu.to_device(s) for s in scs]
    srv = igs.Server(pool_bytes=3 << 30, slots=slots, tile=16)
    sids = [srv.add_scene(d, sh_degree=s.sh_degree) for d, s in zip(devs, scs)]
    reqs = _requests(14, 53, len(scs))
    outs, timings = _serve(srv, sids, reqs)
    stats = srv.stats()
    srv.close()
    assert stats["pool_peak"] <= 3 << 30
    for (s, cam), o, t in zip(reqs, outs, timings):
        alone = _gpu.run_forward(scs[s], cam, tile=16)[3]
        np.testing.assert_array_equal(o.cpu().numpy().astype(np.float64), alone)
        assert t["arrival_ns"] <= t["admit_ns"] <= t["start_ns"] <= t["done_ns"]


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
