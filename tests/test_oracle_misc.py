"""Pins of the oracle's SH basis, activation, L1 loss and Adam.

SH: scipy's complex spherical harmonics converted to the real basis without
Condon-Shortley phase; orthonormality by exact quadrature; the surface gradient
by finite differences on the sphere. Loss and optimiser: torch's l1_loss
autograd and torch.optim.Adam (library routines)."""
import math

import numpy as np
import pytest
import torch
from scipy.special import sph_harm_y

import oracle


def _unit_dirs(n, seed):
    d = np.random.default_rng(seed).normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_sh_matches_scipy():
    d = _unit_dirs(200, 0)
    Y, _ = oracle.sh_basis(3, d)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            k = l * l + l + m
            cy = sph_harm_y(l, abs(m), theta, phi)            # complex, with Condon-Shortley phase
            if m > 0:
                want = math.sqrt(2) * (-1) ** m * cy.real
            elif m < 0:
                want = math.sqrt(2) * (-1) ** m * cy.imag
            else:
                want = cy.real
            np.testing.assert_allclose(Y[:, k], want, atol=1e-13, err_msg=f"l={l} m={m}")


def test_sh_dc_constant():
    Y, dY = oracle.sh_basis(0, _unit_dirs(5, 1))
    np.testing.assert_allclose(Y[:, 0], 1 / (2 * math.sqrt(math.pi)), rtol=1e-15)
    assert np.all(dY == 0)


def test_sh_orthonormal_by_quadrature():
    zs, wz = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phis = 2 * np.pi * np.arange(nphi) / nphi
    Z, P = np.meshgrid(zs, phis, indexing="ij")
    Wt = (wz[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    rxy = np.sqrt(1 - Z ** 2)
    d = np.stack([rxy * np.cos(P), rxy * np.sin(P), Z], axis=-1).reshape(-1, 3)
    Y, _ = oracle.sh_basis(3, d)
    gram = (Y * Wt[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-13)


def test_sh_surface_gradient():
    d = _unit_dirs(50, 2)
    Y, dY = oracle.sh_basis(3, d)
    rng = np.random.default_rng(3)
    h = 1e-6
    for i in range(d.shape[0]):
        tvec = rng.normal(size=3)
        tvec -= (tvec @ d[i]) * d[i]
        tvec /= np.linalg.norm(tvec)
        p = d[i] + h * tvec
        m = d[i] - h * tvec
        Yp, _ = oracle.sh_basis(3, (p / np.linalg.norm(p))[None])
        Ym, _ = oracle.sh_basis(3, (m / np.linalg.norm(m))[None])
        fd = (Yp[0] - Ym[0]) / (2 * h)
        proj = dY[i] - np.outer(dY[i] @ d[i], d[i])          # tangential part of the gradient
        np.testing.assert_allclose(proj @ tvec, fd, atol=1e-7)


def test_activation():
    x = np.linspace(-8, 3, 101).astype(np.float32)
    s, o = oracle.activate(x, x)
    np.testing.assert_array_equal(s, np.exp(x.astype(np.float64)).astype(np.float32))
    np.testing.assert_array_equal(o, (1 / (1 + np.exp(-x.astype(np.float64)))).astype(np.float32))


def test_l1_matches_torch():
    rng = np.random.default_rng(4)
    img = rng.uniform(size=(3, 9, 11))
    tg = rng.uniform(size=(3, 9, 11)).astype(np.float32)
    tg[0, 0, 0] = img[0, 0, 0]                                # a tie: gradient 0 (torch's sign(0) = 0)
    loss, grad = oracle.l1(img, tg)
    ti = torch.tensor(img, requires_grad=True)
    tl = torch.nn.functional.l1_loss(ti, torch.tensor(tg, dtype=torch.float64))
    tl.backward()
    assert loss == pytest.approx(float(tl.detach()), rel=1e-14)
    np.testing.assert_allclose(grad, ti.grad.numpy(), rtol=1e-14)


def test_adam_matches_torch():
    rng = np.random.default_rng(5)
    p0 = rng.normal(size=257)
    p = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    mine, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for t in range(1, 8):
        g = rng.normal(size=257) * (0.1 if t % 2 else 10.0)
        p.grad = torch.tensor(g)
        opt.step()
        mine, m, v = oracle.adam(mine, g, m, v, lr=1e-3, t=t)
        np.testing.assert_allclose(mine, p.detach().numpy(), rtol=1e-12, atol=1e-15)
