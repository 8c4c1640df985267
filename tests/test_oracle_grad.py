"""Pins of the oracle's adjoint (Eq. 3 and the position gradient after it,
through Eq. 4, Eq. 8 and the projection).

Two independent checks: central finite differences of the oracle's own FP64
forward pass (Richardson-extrapolated, steps exactly representable in FP32),
and torch.float64 autograd through a dense renderer written here from the
equations, with the SH basis written out as Cartesian polynomials (a second,
independent derivation of the basis the oracle builds from Legendre polynomials).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from tests._tiny import random_small

A_MIN = float(np.float32(1 / 255))
A_MAX = float(np.float32(0.99))
T_MIN = float(np.float32(1e-4))


def _params(sc):
    return [("means_sigma", sc.means_sigma), ("opacity", sc.opacity), ("color", sc.color)]


def _loss(sc, cam, W, bg):
    out = oracle.render(sc, cam, mode=0, proj64=True, bg=bg, flag_margin=1e-7)
    return float((out["img"] * W).sum()), out["hash"]


def _fd_check(sc, cam, bg=(0.0, 0.0, 0.0), seed=0, rtol=2e-5):
    H, W_ = cam.height, cam.width
    W = np.random.default_rng(seed).normal(size=(3, H, W_))
    g = oracle.backward(sc, cam, W, mode=0, proj64=True, bg=bg)
    analytic = {"means_sigma": np.concatenate([g["d_means"], g["d_sigma"][:, None]], axis=1),
                "opacity": g["d_opac"], "color": g["d_color"]}
    checked = excluded = 0
    scale = max(np.abs(a).max() for a in analytic.values())
    for name, arr in _params(sc):
        flat = arr.reshape(-1)
        an = analytic[name].reshape(-1)
        for j in range(flat.size):
            x0 = flat[j]
            vals, hashes = [], []
            for h in (2.0 ** -16, 2.0 ** -17):
                pair = []
                for sgn in (1, -1):
                    flat[j] = np.float32(x0 + sgn * h)
                    assert float(flat[j]) == float(x0) + sgn * h       # step exact in FP32
                    L, hs = _loss(sc, cam, W, bg)
                    pair.append(L)
                    hashes.append(hs)
                flat[j] = x0
                vals.append((pair[0] - pair[1]) / (2 * h))
            if any(not np.array_equal(hashes[0], hs) for hs in hashes[1:]):
                excluded += 1                                         # a decision flipped: a.e. derivative only
                continue
            fd = (4 * vals[1] - vals[0]) / 3                           # Richardson
            assert abs(fd - an[j]) <= rtol * scale + 1e-6 * abs(an[j]), (name, j, fd, an[j])
            checked += 1
    assert checked >= 0.8 * (checked + excluded)
    return checked


def test_fd_linear_rgb():
    sc, cam = random_small(8, 21, w=20, h=16, spread=0.4, smin=0.05, smax=0.15)
    assert _fd_check(sc, cam, seed=1) > 30


def test_fd_linear_rgb_background():
    sc, cam = random_small(6, 22, w=20, h=16, spread=0.4, smin=0.05, smax=0.15)
    _fd_check(sc, cam, bg=(0.25, 0.5, 0.75), seed=2)


def test_fd_log_params_sh3():
    sc, cam = random_small(5, 23, w=18, h=14, sh_degree=3, log_params=True, spread=0.4, smin=0.05, smax=0.15)
    assert _fd_check(sc, cam, seed=3) > 150


def test_fd_alpha_clamp_active():
    sc, cam = random_small(6, 24, w=18, h=14, spread=0.3, smin=0.08, smax=0.15)
    sc.opacity[:3] = np.float32(0.995)                      # o g > 0.99 near the centres
    _fd_check(sc, cam, seed=4)


# ------------------------------------------------------------- torch pin ----

def _sh_cartesian(deg, d):
    """Real SH without Condon-Shortley phase as Cartesian polynomials (torch)."""
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    c0 = 1 / (2 * math.sqrt(math.pi))
    c1 = math.sqrt(3 / (4 * math.pi))
    out = [torch.full_like(x, c0)]
    if deg >= 1:
        out += [c1 * y, c1 * z, c1 * x]
    if deg >= 2:
        k = math.sqrt(15 / (4 * math.pi))            # 1.0925...
        k0 = math.sqrt(5 / (16 * math.pi))           # 0.3153...
        out += [k * x * y, k * y * z, k0 * (3 * z * z - 1), k * x * z, 0.5 * k * (x * x - y * y)]
    if deg >= 3:
        a = math.sqrt(35 / (32 * math.pi))           # 0.5900...
        b = math.sqrt(105 / (4 * math.pi))          # 2.8906...
        c = math.sqrt(21 / (32 * math.pi))           # 0.4570...
        e = math.sqrt(7 / (16 * math.pi))            # 0.3731...
        out += [a * (3 * x * x * y - y ** 3), b * x * y * z, c * y * (5 * z * z - 1),
                e * (5 * z ** 3 - 3 * z), c * x * (5 * z * z - 1), 0.5 * b * z * (x * x - y * y),
                a * (x ** 3 - 3 * x * y * y)]
    return torch.stack(out, dim=1)


def _torch_render(ms, op, col, cam, sh_degree, log_params, bg):
    R = torch.tensor(cam.R, dtype=torch.float64)
    t = torch.tensor(cam.t, dtype=torch.float64)
    mu = ms[:, :3]
    xc = mu @ R.T + t
    z = xc[:, 2]
    sigma = torch.exp(ms[:, 3]) if log_params else ms[:, 3]
    o = torch.sigmoid(op) if log_params else op
    u = cam.fx * xc[:, 0] / z + cam.cx
    v = cam.fy * xc[:, 1] / z + cam.cy
    s = cam.fx * sigma / z
    n = ms.shape[0]
    if sh_degree < 0:
        rgb = col
    else:
        cc = torch.tensor(cam.center(), dtype=torch.float64)
        d = mu - cc
        d = d / torch.linalg.norm(d, dim=1, keepdim=True)
        Y = _sh_cartesian(sh_degree, d)
        rgb = torch.clamp(torch.einsum("nk,nkc->nc", Y, col.reshape(n, -1, 3)) + 0.5, min=0.0)
    zd = z.detach()
    order = sorted(range(n), key=lambda i: (float(zd[i]), i))
    H, W = cam.height, cam.width
    py, px = torch.meshgrid(torch.arange(H, dtype=torch.float64) + 0.5,
                            torch.arange(W, dtype=torch.float64) + 0.5, indexing="ij")
    T = torch.ones(H, W, dtype=torch.float64)
    C = torch.zeros(3, H, W, dtype=torch.float64)
    alive = torch.ones(H, W, dtype=torch.bool)
    for i in order:
        g = torch.exp(-((px - u[i]) ** 2 + (py - v[i]) ** 2) / (2 * s[i] ** 2))
        a = torch.clamp(o[i] * g, max=A_MAX)
        keep = alive & (a >= A_MIN)
        Tn = T * (1 - a)
        stop = keep & (Tn < T_MIN)
        blend = keep & ~stop
        alive = alive & ~stop
        C = C + torch.where(blend, rgb[i][:, None, None] * a * T, torch.zeros_like(C))
        T = torch.where(blend, Tn, T)
    return C + T * torch.tensor(bg, dtype=torch.float64)[:, None, None]


@pytest.mark.parametrize("case", ["rgb", "sh3_log"])
def test_torch_autograd_matches(case):
    if case == "rgb":
        sc, cam = random_small(12, 31, w=24, h=18, spread=0.5)
    else:
        sc, cam = random_small(12, 32, w=24, h=18, sh_degree=3, log_params=True, spread=0.5)
    bg = (0.25, 0.5, 0.125)
    W = np.random.default_rng(5).normal(size=(3, cam.height, cam.width))
    ms = torch.tensor(sc.means_sigma, dtype=torch.float64, requires_grad=True)
    op = torch.tensor(sc.opacity, dtype=torch.float64, requires_grad=True)
    col = torch.tensor(sc.color, dtype=torch.float64, requires_grad=True)
    img = _torch_render(ms, op, col, cam, sc.sh_degree, sc.log_params, bg)
    (img * torch.tensor(W)).sum().backward()
    g = oracle.backward(sc, cam, W, mode=0, proj64=True, bg=bg)
    np.testing.assert_allclose(g["img"], img.detach().numpy(), atol=1e-12)
    np.testing.assert_allclose(g["d_means"], ms.grad[:, :3].numpy(), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(g["d_sigma"], ms.grad[:, 3].numpy(), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(g["d_opac"], op.grad.numpy(), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(g["d_color"], col.grad.numpy(), rtol=1e-8, atol=1e-10)


def test_lists_mode_gradients_equal_literal():
    sc, cam = random_small(150, 33, w=40, h=30, sh_degree=3, log_params=True, spread=0.8)
    W = np.random.default_rng(6).normal(size=(3, cam.height, cam.width))
    a = oracle.backward(sc, cam, W, mode=0)
    b = oracle.backward(sc, cam, W, mode=1)
    for k in ("d_means", "d_sigma", "d_opac", "d_color"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-15)   # summation order only
