"""Host logic of the renderer's frame pool (no GPU needed: frames are laid out
in host memory here and no kernel runs). The autograd Function leases one frame
per forward; a frame comes back when its backward ran or its graph was freed,
and never while another holder has it."""
import gc

from paper_2403_14244_gb300 import scenes
from paper_2403_14244_gb300.render import Renderer, _FrameLease


def _cam(w=64, h=48):
    return scenes.pinhole((0.0, 0.0, -4.0), w, h, 60.0)


def test_leases_of_one_size_are_distinct_frames():
    r = Renderer(tile=16, device="cpu")
    a = r.lease(100, _cam(), 1024)
    b = r.lease(100, _cam(), 1024)
    assert a is not b and a.leased and b.leased
    shared = r.frame(100, _cam(), 1024)
    assert shared is not a and shared is not b       # the shared frame is not in the pool
    r.release(a)
    c = r.lease(100, _cam(), 1024)
    assert c is a and c.generation == 2              # reused, and its generation moved on
    assert r.lease(100, _cam(64, 40), 1024) is not b  # another size: its own frames


def test_release_of_an_old_generation_is_ignored():
    r = Renderer(tile=16, device="cpu")
    a = r.lease(100, _cam(), 1024)
    gen = a.generation
    r.release(a, gen)
    again = r.lease(100, _cam(), 1024)
    assert again is a
    r.release(a, gen)                                # a stale holder: the new lease stands
    assert a.leased
    r.release(a)
    r.release(a)                                     # releasing twice is harmless
    assert r._free[(100, 64, 48)] == [a]


def test_too_small_pooled_frames_are_dropped():
    r = Renderer(tile=16, device="cpu")
    a = r.lease(100, _cam(), 1024)
    r.release(a)
    b = r.lease(100, _cam(), 4096)
    assert b is not a and b.capacity == 4096
    assert r._free.get((100, 64, 48), []) == []


def test_lease_holder_returns_the_frame_when_collected():
    r = Renderer(tile=16, device="cpu")
    f = r.lease(100, _cam(), 1024)
    holder = _FrameLease(r, f)
    assert f.leased
    del holder
    gc.collect()
    assert not f.leased and r.lease(100, _cam(), 1024) is f
