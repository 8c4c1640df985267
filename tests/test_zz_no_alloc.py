"""igs_sort_depth_noalloc, called through the C ABI, against igs_bin_sort.

Some callers of this library cannot allocate device memory around a call: a
host whose device memory all belongs to its own allocator, or a loop that must
not call cudaMalloc/cudaFree because they can synchronise the device.
igs_sort_depth_noalloc serves them: it orders depth keys front to back like
igs_bin_sort does for a frame, with its scratch in a fixed array inside the
library. This file is collected last on purpose, and its tests
pass both on their own in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest
import torch

from paper_2403_14244_gb300 import igs, scenes
from tests import _gpu

pytestmark = pytest.mark.gpu


def _bin_sort_order(sc, cam):
    """depth keys and front-to-back order from the existing entry point."""
    r, f, scene, img = _gpu.run_forward(sc, cam)
    return f.depth_key().clone(), f.order().clone()


def test_noalloc_order_matches_bin_sort_on_two_calls_in_a_row():
    # 700,001 Gaussians (a ragged last block), every fourth one duplicated so that
    # equal depths occur and the tie rule (index order) is exercised
    sc = scenes.clustered_scene(700_001, 31)
    sc.means_sigma[3::4] = sc.means_sigma[2::4][: sc.means_sigma[3::4].shape[0]]
    cams = [scenes.pinhole((0.3, -0.2, -3.7), 1280, 720, 1000.0),
            scenes.pinhole((-2.0, 0.5, 0.6), 640, 360, 560.0)]      # the second sees only part of the scene
    for cam in cams:
        dk, want = _bin_sort_order(sc, cam)
        got = torch.full_like(want, -1)
        igs.sort_depth_noalloc(dk, got)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        assert (dk.cpu().numpy().view(np.uint32) == 0xFFFFFFFF).any() or cam is cams[0]


def test_noalloc_rejects_more_keys_than_its_scratch_holds():
    dk = torch.zeros((1 << 20) + 1, dtype=torch.int32, device="cuda")
    out = torch.empty_like(dk)
    with pytest.raises(igs.IgsError) as e:
        igs.sort_depth_noalloc(dk, out)
    assert e.value.status == igs.ERR_INVALID_ARG
