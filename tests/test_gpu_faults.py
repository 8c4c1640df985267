"""Failure detection on the GPU without a fault: a bounded device wait is made
to run out (one block of the first depth-sort pass never publishes its digit
counts, a test switch of the library), and the frame must report
IGS_ERR_DEVICE_TIMEOUT, abort (the blend leaves the image untouched), and
leave the context usable (the next frame renders the same image as before)."""
import time

import pytest
import torch

from paper_2403_14244_gb300 import igs, scenes
from paper_2403_14244_gb300.render import Renderer

pytestmark = pytest.mark.gpu


def test_lost_lookback_times_out_and_aborts_the_frame():
    _, cam = scenes.workload_forward_4k()
    sc = scenes.uniform_scene(20000, 61)          # five blocks in each depth-sort pass
    scene = igs.Scene.from_numpy(sc, "cuda")
    r = Renderer(tile=16)
    ref, _ = r.run_forward(scene, cam, check=True)
    ref = ref.clone()
    img = torch.full_like(ref, 7.0)
    igs.debug_silence_lookback_once()
    t0 = time.perf_counter()
    _, f = r.run_forward(scene, cam, img=img, check=False)
    st, info = igs.frame_status(f)
    waited = time.perf_counter() - t0
    assert st == igs.ERR_DEVICE_TIMEOUT and info[2] == igs.ERR_DEVICE_TIMEOUT
    assert waited < 30.0                            # bounded: the waits gave up
    assert torch.all(img == 7.0)                    # aborted frame: the blend wrote nothing
    again, f2 = r.run_forward(scene, cam, check=True)
    torch.cuda.synchronize()
    assert igs.frame_status(f2)[0] == igs.OK
    assert torch.equal(again, ref)                  # the context and the library work as before
