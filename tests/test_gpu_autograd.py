"""The torch.autograd.Function over the CUDA path (render.IGSRender): gradients
reached through loss.backward(), against the FP64 oracle's analytic adjoint
(Eq. 3 and the position gradient after it, through Eq. 4 and Eq. 8) and against
central differences of the oracle's FP64 forward."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2403_14244_gb300.render import Renderer, render
from tests import _gpu
from tests._tiny import random_small

pytestmark = pytest.mark.gpu


def _leaves(sc):
    return [torch.from_numpy(a).cuda().requires_grad_(True) for a in (sc.means_sigma, sc.opacity, sc.color)]


def _oracle_grads(sc, cam, W):
    g = oracle.backward(sc, cam, W, mode=1)
    return np.concatenate([g["d_means"], g["d_sigma"][:, None]], 1), g["d_opac"], g["d_color"]


def _check(leaves, want):
    for name, t, w in zip(("means_sigma", "opacity", "color"), leaves, want):
        _gpu.grad_close(t.grad.cpu().numpy(), w, name)


@pytest.mark.parametrize("sh_degree,log_params", [(-1, False), (3, True)])
def test_backward_through_autograd_one_view(sh_degree, log_params):
    sc, cam = random_small(300, 61, w=80, h=60, sh_degree=sh_degree, log_params=log_params, spread=0.8)
    W = np.random.default_rng(11).normal(size=(3, cam.height, cam.width))
    r = Renderer(tile=16, sh_degree=sh_degree, param_mode=int(log_params))
    leaves = _leaves(sc)
    img = render(*leaves, r, cam)
    (img * torch.from_numpy(W.astype(np.float32)).cuda()).sum().backward()
    _check(leaves, _oracle_grads(sc, cam, W))


def test_two_views_of_one_size_in_one_loss():
    """Two renders of the same image size summed into one loss before backward():
    each backward must walk its own view's lists (the gradient is the sum of the
    two oracle gradients), and a third view of another size joins the sum."""
    sc, cam = random_small(400, 62, w=96, h=64, spread=0.8)
    cam2 = dataclasses.replace(cam, t=(np.asarray(cam.t, np.float32) + np.float32([0.15, -0.1, 0.2])))
    cam3 = dataclasses.replace(cam, width=72, height=56, cx=36.0, cy=28.0)
    rng = np.random.default_rng(12)
    Ws = [rng.normal(size=(3, c.height, c.width)) for c in (cam, cam2, cam3)]
    r = Renderer(tile=16)
    leaves = _leaves(sc)
    loss = 0
    for c, W in zip((cam, cam2, cam3), Ws):
        loss = loss + (render(*leaves, r, c) * torch.from_numpy(W.astype(np.float32)).cuda()).sum()
    loss.backward()
    refs = [_oracle_grads(sc, c, W) for c, W in zip((cam, cam2, cam3), Ws)]
    _check(leaves, [sum(parts) for parts in zip(*refs)])
    # the frames went back to the pool: a new pair of renders reuses them
    assert sum(len(v) for v in r._free.values()) == 3


def test_second_backward_after_reuse_is_refused():
    """retain_graph: a second backward works while the frame is untouched, and
    is refused (not silently wrong) once a later forward has reused it."""
    sc, cam = random_small(200, 63, w=64, h=48, spread=0.7)
    W = torch.from_numpy(np.random.default_rng(13).normal(size=(3, cam.height, cam.width)).astype(np.float32)).cuda()
    r = Renderer(tile=16)
    leaves = _leaves(sc)
    loss = (render(*leaves, r, cam) * W).sum()
    loss.backward(retain_graph=True)
    g1 = leaves[2].grad.clone()
    loss.backward(retain_graph=True)
    torch.testing.assert_close(leaves[2].grad, 2 * g1, rtol=1e-5, atol=1e-7)
    render(*[t.detach() for t in leaves], r, cam)  # leases (and overwrites) the same frame
    with pytest.raises(RuntimeError, match="reused"):
        loss.backward()


def _fd_grads(sc, cam, W, names_idx):
    """Richardson-extrapolated central differences of sum(W * img) for the
    oracle's FP64 forward (FP64 disc), steps exact in FP32; entries whose step
    flips a cutoff or stop decision somewhere are returned as NaN."""
    out = {}
    for name, arr in (("means_sigma", sc.means_sigma), ("opacity", sc.opacity), ("color", sc.color)):
        flat = arr.reshape(-1)
        fd = np.full(flat.size, np.nan)
        for j in names_idx(name, flat.size):
            x0 = flat[j]
            vals, hashes = [], []
            for h in (2.0 ** -15, 2.0 ** -16):
                pair = []
                for sgn in (1, -1):
                    flat[j] = np.float32(x0 + sgn * h)
                    o = oracle.render(sc, cam, mode=0, proj64=True, flag_margin=1e-7)
                    pair.append(float((o["img"] * W).sum()))
                    hashes.append(o["hash"])
                flat[j] = x0
                vals.append((pair[0] - pair[1]) / (2 * h))
            if all(np.array_equal(hashes[0], hs) for hs in hashes[1:]):
                fd[j] = (4 * vals[1] - vals[0]) / 3
        out[name] = fd.reshape(arr.shape)
    return out


@pytest.mark.parametrize("n,sh_degree,log_params", [(48, -1, False), (12, 3, True)])
def test_autograd_against_oracle_finite_differences(n, sh_degree, log_params):
    """Central differences in FP64 through the oracle's forward, on a scene of at
    most 64 Gaussians, against the gradient the CUDA adjoint returns through
    loss.backward(). The GPU composites FP32 discs, the differences FP64 ones,
    so the bound is the FP32 one of the adjoint parity tests (1e-3)."""
    sc, cam = random_small(n, 64 + n, w=28, h=22, sh_degree=sh_degree, log_params=log_params, spread=0.45,
                           smin=0.05, smax=0.15)
    W = np.random.default_rng(14).normal(size=(3, cam.height, cam.width))
    r = Renderer(tile=8, sh_degree=sh_degree, param_mode=int(log_params))
    leaves = _leaves(sc)
    (render(*leaves, r, cam) * torch.from_numpy(W.astype(np.float32)).cuda()).sum().backward()
    fd = _fd_grads(sc, cam, W, lambda name, size: range(size))
    checked = 0
    scale = max(np.nanmax(np.abs(v)) for v in fd.values())
    for name, t in zip(("means_sigma", "opacity", "color"), leaves):
        got = t.grad.cpu().numpy().astype(np.float64)
        ok = ~np.isnan(fd[name])
        err = np.abs(got[ok] - fd[name][ok])
        bound = 1e-3 * np.abs(fd[name][ok]) + 1e-3 * scale
        assert (err <= bound).all(), f"{name}: worst {np.max(err - bound):.3e} over the bound"
        checked += int(ok.sum())
    total = sum(v.size for v in fd.values())
    assert checked >= 0.8 * total, (checked, total)
