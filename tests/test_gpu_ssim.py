"""GPU parity of the loss of Sec. 3 with its SSIM term, (1 - lambda) L1 +
lambda (1 - SSIM), and its image gradient, against the oracle's FP64 values
(pinned by scipy's Gaussian filter, closed forms, finite differences and torch
autograd in the CPU tests).

Tolerances, from the FP32 arithmetic: the window sums and the variances
E[x^2] - mx^2 carry relative errors of a few 1e-7 of mx^2, divided by
sxx + syy + C2 >= C2 = 9e-4 in the partials, so the gradient is checked to
1e-3 relative plus 2e-4 of its largest entry, the loss and the mean SSIM to
1e-5 (they are sums of per-tile partials added in any order)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_14244_gb300 import igs

pytestmark = pytest.mark.gpu


def _smooth(shape, rng):
    """Low-frequency image in [0, 1] with flat regions (low local variance)."""
    C, H, W = shape
    yy, xx = np.meshgrid(np.arange(H) / max(H, 1), np.arange(W) / max(W, 1), indexing="ij")
    out = np.empty(shape)
    for c in range(C):
        f = rng.uniform(0.5, 4.0, size=4)
        ph = rng.uniform(0, 2 * np.pi, size=4)
        v = 0.5 + 0.2 * np.sin(2 * np.pi * f[0] * xx + ph[0]) * np.cos(2 * np.pi * f[1] * yy + ph[1])
        v += 0.1 * np.sin(2 * np.pi * (f[2] * xx + f[3] * yy) + ph[2])
        out[c] = np.clip(v, 0.0, 1.0)
    return out


def _inputs(shape, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        x, y = rng.random(shape), rng.random(shape)
    else:
        x = _smooth(shape, rng)
        y = np.clip(x + 0.02 * rng.normal(size=shape), 0.0, 1.0)
    return x.astype(np.float32), y.astype(np.float32)


def _gpu(x, y, lam):
    tx, ty = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    loss = torch.zeros(1, device="cuda")
    ssim = torch.zeros(1, device="cuda")
    grad = torch.empty_like(tx)
    work = torch.empty(igs.ssim_work_bytes(*x.shape) // 4, device="cuda")
    igs.l1_ssim_loss(tx, ty, lam, loss, grad, work, ssim=ssim)
    torch.cuda.synchronize()
    return loss.item(), ssim.item(), grad.cpu().numpy()


def _check(x, y, lam):
    loss, ssim, g = _gpu(x, y, lam)
    want, s_ref, g_ref = oracle.l1_ssim(x.astype(np.float64), y.astype(np.float64), lam=lam)
    assert loss == pytest.approx(want, rel=1e-5, abs=1e-6)
    assert ssim == pytest.approx(s_ref, rel=1e-5, abs=1e-6)
    err = np.abs(g.astype(np.float64) - g_ref)
    bound = 1e-3 * np.abs(g_ref) + 2e-4 * np.abs(g_ref).max()
    assert np.all(err <= bound), f"worst {np.max(err - bound):.3e} over bound, max|g| {np.abs(g_ref).max():.3e}"
    return g, g_ref


@pytest.mark.parametrize("kind", ["uniform", "smooth"])
@pytest.mark.parametrize("shape", [(3, 100, 75), (1, 33, 65), (3, 64, 64), (2, 5, 3), (1, 1, 1), (3, 1, 40)])
@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_l1_ssim_matches_oracle(shape, kind, lam):
    x, y = _inputs(shape, kind, sum(shape) * 10 + len(kind))
    _check(x, y, lam)


@pytest.mark.parametrize("kind", ["uniform", "smooth"])
def test_l1_ssim_training_image_size(kind):
    # the 1297 x 840 RGB images of the training workload (ragged 32 x 32 tiles on both axes)
    x, y = _inputs((3, 840, 1297), kind, 7)
    _check(x, y, 0.2)


def test_identical_images():
    x, _ = _inputs((3, 70, 90), "smooth", 3)
    loss, ssim, g = _gpu(x, x, 1.0)
    assert ssim == pytest.approx(1.0, abs=2e-6)
    assert abs(loss) < 2e-6
    assert np.abs(g).max() < 1e-3 / x.size


def test_lambda_zero_is_the_l1_kernel():
    x, y = _inputs((3, 50, 61), "uniform", 4)
    loss, _, g = _gpu(x, y, 0.0)
    tx, ty = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    l1 = torch.zeros(1, device="cuda")
    g1 = torch.empty_like(tx)
    igs.l1_loss(tx, ty, l1, g1)
    np.testing.assert_allclose(g, g1.cpu().numpy(), rtol=1e-6, atol=0)
    assert loss == pytest.approx(l1.item(), rel=1e-5)


def test_bad_arguments_raise():
    x = torch.zeros(3, 8, 8, device="cuda")
    loss = torch.zeros(1, device="cuda")
    work = torch.empty(igs.ssim_work_bytes(3, 8, 8) // 4, device="cuda")
    with pytest.raises(igs.IgsError):
        igs.l1_ssim_loss(x, x, 1.5, loss, torch.empty_like(x), work)
    with pytest.raises(ValueError):
        igs.l1_ssim_loss(x, x, 0.2, loss, torch.empty_like(x), work[:10])
    assert igs.ssim_work_bytes(0, 8, 8) == 0


def test_train_step_with_ssim_matches_oracle():
    """One training step with the paper's loss (lambda = 0.2): the gradient the
    step writes (unfused path) against the oracle's render -> L1 + SSIM ->
    adjoint chain in FP64."""
    from paper_2403_14244_gb300 import scenes
    from paper_2403_14244_gb300.render import TrainStep
    from tests import _gpu as g
    from tests._tiny import random_small

    sc, cam = random_small(500, 46, w=96, h=64, sh_degree=3, log_params=True, spread=0.8)
    target = scenes.target_image(cam.width, cam.height, 11)
    ref_fwd = oracle.render(sc, cam, mode=1)
    loss_ref, _, G = oracle.l1_ssim(ref_fwd["img"], target.astype(np.float64), lam=0.2)
    ref = oracle.backward(sc, cam, G, mode=1)
    ts = TrainStep(torch.from_numpy(sc.means_sigma).cuda(), torch.from_numpy(sc.opacity).cuda(),
                   torch.from_numpy(sc.color).cuda(), sh_degree=3, lr=1e-3, fused=False, ssim_lambda=0.2)
    ts.step(cam, torch.from_numpy(target).cuda(), check=True)
    torch.cuda.synchronize()
    assert float(ts.loss) == pytest.approx(loss_ref, rel=1e-4)
    g.grad_close(ts.g_ms.cpu().numpy(), np.concatenate([ref["d_means"], ref["d_sigma"][:, None]], 1), "means_sigma")
    g.grad_close(ts.g_op.cpu().numpy(), ref["d_opac"], "opacity")
    g.grad_close(ts.g_col.cpu().numpy(), ref["d_color"], "color")


def test_misaligned_work_is_rejected():
    x = torch.rand(3, 16, 16, device="cuda")
    loss = torch.zeros(1, device="cuda")
    work = torch.empty(igs.ssim_work_bytes(3, 16, 16) // 4 + 4, device="cuda")
    with pytest.raises(igs.IgsError):
        igs.l1_ssim_loss(x, x, 0.2, loss, torch.empty_like(x), work[1:])
