"""Helpers for the GPU parity tests: run the CUDA path through the C ABI on a
numpy scene and bring the results back to the host."""
import numpy as np
import torch

from paper_2403_14244_gb300 import igs
from paper_2403_14244_gb300.render import Renderer


def to_device(sc):
    return igs.Scene.from_numpy(sc, "cuda")


def run_forward(sc, cam, tile=16, bg=(0.0, 0.0, 0.0), capacity=None, footprint=0):
    """project + bin_sort + render_fwd; returns (renderer, frame, scene, img numpy)."""
    r = Renderer(tile=tile, sh_degree=sc.sh_degree, param_mode=int(sc.log_params), bg=bg, footprint=footprint)
    scene = to_device(sc)
    if capacity is not None:
        r._cap_hint[(scene.n, cam.width, cam.height)] = capacity
    img, f = r.run_forward(scene, cam, check=True)
    torch.cuda.synchronize()
    return r, f, scene, img.cpu().numpy().astype(np.float64)


def frame_keys(f):
    st, info = igs.frame_status(f)
    assert st == igs.OK, st
    M = info[0]
    keys = igs.export_keys(f)[:M].cpu().numpy().view(np.uint64)
    vals = f.vals(M).cpu().numpy().view(np.uint32)
    ranges = f.ranges().cpu().numpy().view(np.uint32)
    return keys, vals, ranges, info


def compare_images(got, want, flag, atol=2e-4, max_flag_frac=1e-3):
    """|got - want| <= atol per channel outside the flagged pixels; flagged
    pixels (a cutoff or stop decision within the oracle's margin) are counted."""
    ok = flag == 0
    assert flag.mean() <= max_flag_frac, f"flagged fraction {flag.mean():.2e}"
    err = np.abs(got - want)[:, ok]
    assert err.size == 0 or err.max() <= atol, f"max err {err.max():.3e} at {np.unravel_index(err.argmax(), err.shape)}"
    return float(err.max()) if err.size else 0.0


def grad_close(got, want, name, rel_norm=1e-3, elem_rel=1e-3, elem_abs_frac=1e-3):
    """Per parameter block: relative L2 error <= rel_norm, and elementwise
    |g - g_ref| <= elem_rel |g_ref| + elem_abs_frac max|g_ref|."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    nrm = np.linalg.norm(want)
    if nrm == 0:
        assert np.abs(got).max() == 0, name
        return 0.0
    rel = np.linalg.norm(got - want) / nrm
    assert rel <= rel_norm, f"{name}: relative L2 error {rel:.3e}"
    bound = elem_rel * np.abs(want) + elem_abs_frac * np.abs(want).max()
    bad = np.abs(got - want) > bound
    assert not bad.any(), f"{name}: {bad.sum()} elements out of bound, worst at {np.argmax(np.abs(got - want) - bound)}"
    return float(rel)
