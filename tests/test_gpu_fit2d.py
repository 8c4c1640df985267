"""GPU parity of the paper's 2D experiment (Sec. 3) against the oracle: the
additive render (the FP32 support decision is canonical on both sides, values
within FP32 rounding), the particle gradient (P19's gradient tolerance), the
QuadTree initialisation (bit for bit: the statistics are exact integers), the
per-slot Adam step, one full fitting iteration, and graph replay against eager
steps."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_14244_gb300 import igs, scenes
from paper_2403_14244_gb300.fit2d import DEFAULT_LR, Fit2D
from tests import _gpu

pytestmark = pytest.mark.gpu


def _render(p, D, W, H):
    tp = torch.from_numpy(np.ascontiguousarray(p, np.float32)).cuda()
    img = torch.empty((3, H, W), device="cuda")
    igs.fit2d_render(tp, D, img)
    torch.cuda.synchronize()
    return img.cpu().numpy()


def _img_close(got, want):
    # each pixel sums terms A g with g from ex2.approx and FP32 exponents: a few 1e-7 relative per term
    scale = max(1.0, float(np.abs(want).max()))
    np.testing.assert_allclose(got, want, rtol=2e-5, atol=2e-5 * scale)


@pytest.mark.parametrize("k,W,H,D", [(1, 40, 30, 9.0), (37, 48, 40, 3.0), (300, 130, 97, 15.0), (300, 64, 64, 50.0),
                                     (1000, 256, 256, 15.0), (700, 100, 120, float("inf")), (0, 33, 17, 5.0)])
def test_render_matches_oracle(k, W, H, D):
    p = scenes.fit2d_particles(k, max(W, H), 10 + k, sigma=(0.7, 20.0))
    _img_close(_render(p, D, W, H), oracle.fit2d_render(p, D, W, H))


def test_render_support_edge_is_exact():
    # particles at fractional positions with D chosen so many pixels sit within rounding of the boundary
    rng = np.random.default_rng(3)
    p = np.zeros((64, 8), np.float32)
    p[:, 0:2] = rng.integers(5, 59, size=(64, 2)) + rng.choice([0.0, 0.5, 0.25, 0.125], size=(64, 2))
    p[:, 2] = np.log(50.0)        # wide kernels: the cutoff, not the Gaussian, decides
    p[:, 3:6] = 1.0
    for D in (3.0, np.sqrt(8.0), 5.0, 7.0710678):
        got, want = _render(p, D, 64, 64), oracle.fit2d_render(p, D, 64, 64)
        # reached pixels get ~1 per particle here, unreached exactly 0: the decisions agree
        np.testing.assert_array_equal(got[0] > 0, want[0] > 0)
        _img_close(got, want)


@pytest.mark.parametrize("k,W,H,D", [(37, 48, 40, 6.0), (300, 130, 97, 15.0), (500, 128, 128, 50.0)])
def test_backward_matches_oracle(k, W, H, D):
    p = scenes.fit2d_particles(k, max(W, H), 20 + k, sigma=(0.7, 15.0))
    G = np.random.default_rng(k).normal(size=(3, H, W)).astype(np.float32)
    tp = torch.from_numpy(p).cuda()
    grad = torch.full((k, 8), 7.0, device="cuda")   # overwritten
    igs.fit2d_backward(tp, D, torch.from_numpy(G).cuda(), grad)
    torch.cuda.synchronize()
    got = grad.cpu().numpy()
    want = oracle.fit2d_backward(p, D, G)
    assert np.all(got[:, 6:] == 0)
    for j, name in enumerate(("mu_x", "mu_y", "log_sigma", "A_r", "A_g", "A_b")):
        _gpu.grad_close(got[:, j], want[:, j], name)


def _qt_gpu(img, k_max, min_cell):
    S = img.shape[1]
    ti = torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda()
    out = torch.full((k_max, 8), -1.0, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    work = torch.empty(igs.quadtree_work_bytes(S, min_cell), dtype=torch.uint8, device="cuda")
    igs.quadtree_init(ti, k_max, min_cell, out, cnt, work)
    torch.cuda.synchronize()
    n = int(cnt.item())
    return out[:n].cpu().numpy()


@pytest.mark.parametrize("S,k_max,min_cell,seed", [(64, 100, 2, 1), (128, 334, 3, 2), (512, 1000, 3, 6),
                                                   (512, 2000, 7, 6), (512, 2000, 1, 6), (32, 10000, 1, 3),
                                                   (256, 1, 4, 4), (16, 7, 32, 5), (1, 5, 1, 2)])
def test_quadtree_bit_exact(S, k_max, min_cell, seed):
    img = scenes.fit2d_image(S, seed) if S > 1 else np.full((3, 1, 1), 0.3, np.float32)
    got = _qt_gpu(img, k_max, min_cell)
    want = oracle.quadtree_init(img, k_max, min_cell)
    assert got.shape == want.shape
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))


def test_quadtree_ties_bit_exact():
    # constant and blocky images: many equal errors, decided by level, row, column
    img = np.zeros((3, 64, 64), np.float32)
    img[:, :32, 32:] = 0.5
    img[1, 40:, :20] = 0.25
    for k_max in (4, 7, 22, 100, 1365):
        got, want = _qt_gpu(img, k_max, 2), oracle.quadtree_init(img, k_max, 2)
        np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))
    flat = np.full((3, 32, 32), 0.7, np.float32)
    np.testing.assert_array_equal(_qt_gpu(flat, 40, 1).view(np.uint32), oracle.quadtree_init(flat, 40, 1).view(np.uint32))


def test_adam_per_slot_matches_oracle():
    rng = np.random.default_rng(5)
    k = 1001
    p0 = rng.normal(size=(k, 8)).astype(np.float32)
    p0[:, 6:] = 0
    p, m, v = torch.from_numpy(p0).cuda(), torch.zeros(k, 8, device="cuda"), torch.zeros(k, 8, device="cuda")
    state = torch.zeros(2, dtype=torch.int32, device="cuda")
    lr = DEFAULT_LR
    rp, rm, rv = p0.astype(np.float64), np.zeros((k, 8)), np.zeros((k, 8))
    for t in range(1, 6):
        g = (rng.normal(size=(k, 8)) * (0.01 if t % 2 else 3.0)).astype(np.float32)
        g[:, 6:] = 0
        igs.fit2d_adam(p, torch.from_numpy(g).cuda(), m, v, lr, state)
        for j in range(8):
            rp[:, j], rm[:, j], rv[:, j] = oracle.adam(rp[:, j], g[:, j], rm[:, j], rv[:, j], lr=lr[j], t=t)
    torch.cuda.synchronize()
    assert state.cpu().tolist() == [5, 0]
    np.testing.assert_allclose(p.cpu().numpy(), rp, rtol=0, atol=2e-6 * 200)   # lr up to 0.2: scale the FP32 ulp
    np.testing.assert_allclose(m.cpu().numpy(), rm, rtol=1e-5, atol=4 * np.spacing(np.float32(0.3)))


def test_fit_iteration_matches_oracle():
    S, D, lam = 64, 9.0, 0.2
    target = scenes.fit2d_image(S, 9)
    f = Fit2D(torch.from_numpy(target).cuda(), 200, D, min_cell=2, lam=lam)
    p0 = f.particles.cpu().numpy()
    np.testing.assert_array_equal(p0.view(np.uint32), oracle.quadtree_init(target, 200, 2).view(np.uint32))
    f.step()
    torch.cuda.synchronize()
    img = oracle.fit2d_render(p0, D, S, S)
    loss_ref, _, G = oracle.l1_ssim(img, target.astype(np.float64), lam=lam)
    g_ref = oracle.fit2d_backward(p0, D, G)
    assert float(f.loss) == pytest.approx(loss_ref, rel=1e-4)
    got_g = f.grad.cpu().numpy()
    for j in range(6):
        _gpu.grad_close(got_g[:, j], g_ref[:, j], f"slot {j}")
    # the first Adam step moves each parameter by lr * sign(g) where |g| is not tiny
    p1 = f.particles.cpu().numpy()
    for j in range(6):
        moved = np.abs(g_ref[:, j]) > 1e-2 * np.abs(g_ref[:, j]).max()
        np.testing.assert_allclose(p1[moved, j] - p0[moved, j], -DEFAULT_LR[j] * np.sign(g_ref[moved, j]),
                                   rtol=1e-3, atol=1e-6)


def test_graph_replay_matches_eager_and_loss_falls():
    S = 128
    target = torch.from_numpy(scenes.fit2d_image(S, 10)).cuda()
    a = Fit2D(target, 334, 15.0, min_cell=3)
    b = Fit2D(target, 334, 15.0, min_cell=3)
    a.capture(inner=10)            # one eager step, then 10 captured
    a.run(40)
    for _ in range(41):
        b.step()
    torch.cuda.synchronize()
    assert a.steps_done() == b.steps_done() == 41
    # the adjoint's atomics add tiles in any order, so runs agree to rounding, not bit for bit
    assert float(a.loss) == pytest.approx(float(b.loss), rel=1e-3)
    close = np.isclose(a.particles.cpu().numpy(), b.particles.cpu().numpy(), rtol=1e-3, atol=1e-3)
    assert close.mean() > 0.99
    first = Fit2D(target, 334, 15.0, min_cell=3)
    first.step()
    torch.cuda.synchronize()
    assert float(a.loss) < 0.7 * float(first.loss)


def test_bad_arguments_raise():
    p = torch.zeros(4, 8, device="cuda")
    img = torch.empty(3, 8, 8, device="cuda")
    with pytest.raises(igs.IgsError):
        igs.fit2d_render(p, 0.0, img)
    with pytest.raises(igs.IgsError):
        igs.fit2d_render(p[:, :].reshape(-1)[1:9].reshape(1, 8), 3.0, img)   # misaligned
    with pytest.raises(igs.IgsError):
        igs.quadtree_init(torch.zeros(3, 48, 48, device="cuda"), 10, 2, p, torch.zeros(1, dtype=torch.int32,
                          device="cuda"), torch.empty(1024, dtype=torch.uint8, device="cuda"))
    assert igs.quadtree_work_bytes(48, 2) == 0


# ------------------------------------------------------------ densify/prune --

def test_grad_accum_bit_exact():
    rng = np.random.default_rng(31)
    g = rng.normal(size=(3000, 8)).astype(np.float32) * np.float32(1e-2)
    g[::17, :2] = 0.0
    a0 = rng.random(3000).astype(np.float32)
    acc = torch.from_numpy(a0).cuda()
    igs.fit2d_grad_accum(torch.from_numpy(g).cuda(), acc)
    igs.fit2d_grad_accum(torch.from_numpy(g[::-1].copy()).cuda(), acc)
    want = oracle.fit2d_grad_accum(g[::-1], oracle.fit2d_grad_accum(g, a0))
    np.testing.assert_array_equal(acc.cpu().numpy(), want)


def _densify_inputs(k, seed):
    p = scenes.fit2d_particles(k, 256, seed, sigma=(0.5, 16.0))
    rng = np.random.default_rng(seed + 1)
    p[rng.random(k) < 0.2, 3:6] *= np.float32(0.02)        # faint: below tau_a
    if k > 3:
        p[1, 3] = np.nan                                    # a NaN first amplitude keeps its particle
        p[2, 3:6] = -0.9                                    # |A| counts, not A
    m = rng.normal(size=(k, 8)).astype(np.float32)
    v = rng.random((k, 8)).astype(np.float32)
    acc = (rng.random(k) * 2.0).astype(np.float32)
    if k > 5:
        acc[5] = np.nan                                     # never a candidate
    return p, m, v, acc


@pytest.mark.parametrize("k,capacity", [(0, 16), (1, 8), (1500, 6000), (1500, 1500), (5000, 9000), (5000, 3000),
                                        (5000, 100), (4096, 4096 * 4)])
def test_densify_bit_exact(k, capacity):
    p, m, v, acc = _densify_inputs(k, 40 + k)
    n_it, tau_a, tau_g, lsm = 7, 0.05, 0.15, float(np.log(1.5))
    want_p, want_m, want_v = oracle.fit2d_densify(p, m, v, acc, n_it, tau_a, tau_g, lsm, capacity)
    t = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (p, m, v, acc)]
    out = torch.full((capacity, 8), 3.0, device="cuda")
    om, ov = torch.full_like(out, 3.0), torch.full_like(out, 3.0)
    count = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    igs.fit2d_densify(*t, n_it, tau_a, tau_g, lsm, out, om, ov, count)
    n = int(count.item())
    assert n == want_p.shape[0]
    np.testing.assert_array_equal(out[:n].cpu().numpy(), want_p)
    np.testing.assert_array_equal(om[:n].cpu().numpy(), want_m)
    np.testing.assert_array_equal(ov[:n].cpu().numpy(), want_v)
    assert torch.all(out[n:] == 3.0)                         # nothing written past the count


def test_densify_rejects_overlap_and_bad_args():
    p = torch.zeros((16, 8), device="cuda")
    acc = torch.zeros(16, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros((32, 8), device="cuda")
    with pytest.raises(igs.IgsError):
        igs.fit2d_densify(p, p, p, acc, 1, 0.1, 0.1, 0.0, out, p, out, count)   # out_m is an input
    with pytest.raises(igs.IgsError):
        igs.fit2d_densify(p, p, p, acc, 0, 0.1, 0.1, 0.0, out, out.clone(), out.clone(), count)


def test_fit2d_driver_densify_matches_oracle():
    img = torch.from_numpy(scenes.fit2d_image(128, 6)).cuda()
    f = Fit2D(img, k_max=100, D=15.0, min_cell=3)
    f.track_grad_norm()
    for _ in range(5):
        f.step()
    f.run(20)                                              # graph replays sum the statistic too
    assert f.accum_iters == 5 + 1 + 20                     # 5 eager, 1 eager at capture, 2 replays of 10
    p, m, v, acc = (x.cpu().numpy() for x in (f.particles, f.m, f.v, f.accum))
    n_it = f.accum_iters
    tau_g = float(np.median(acc)) / n_it
    want_p, want_m, want_v = oracle.fit2d_densify(p, m, v, acc, n_it, 0.02, tau_g, 0.0, 400)
    k = f.densify(0.02, tau_g, 0.0, 400)
    assert k == want_p.shape[0] and k > p.shape[0]
    np.testing.assert_array_equal(f.particles.cpu().numpy(), want_p)
    np.testing.assert_array_equal(f.m.cpu().numpy(), want_m)
    np.testing.assert_array_equal(f.v.cpu().numpy(), want_v)
    assert float(f.accum.abs().sum()) == 0.0 and f.accum_iters == 0
    f.run(20)                                              # continues with the new particle set
    torch.cuda.synchronize()
    _img_close(f.render().cpu().numpy(), oracle.fit2d_render(f.particles.cpu().numpy(), 15.0, 128, 128))
