"""GPU parity of the densify / prune pass of the 3D Gaussians (Sec. 3.2:
deletion below a threshold, division; Sec. 2.5; the Octree of Sec. 3.1 as the
division pattern) against the oracle: the per-step statistic and the
keep / delete / divide pass bit for bit (both sides take every decision on the
same FP32 values), over several blocks, both parameterisations, RGB and SH
colour, capacity limits and NaN inputs; and the training step's use of it."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_14244_gb300 import igs, scenes
from paper_2403_14244_gb300.render import TrainStep
from tests._tiny import random_small

pytestmark = pytest.mark.gpu


def _state(n, C, seed, param_mode):
    rng = np.random.default_rng(seed)
    ms = np.zeros((n, 4), np.float32)
    ms[:, :3] = rng.uniform(-1, 1, (n, 3))
    sig = np.exp(rng.uniform(np.log(0.005), np.log(0.05), n))
    ms[:, 3] = np.log(sig) if param_mode == 1 else sig
    op = (rng.normal(0, 1.5, n) if param_mode == 1 else rng.uniform(0.0, 1.0, n)).astype(np.float32)
    col = rng.normal(0, 0.3, (n, C)).astype(np.float32)
    m = [rng.normal(0, 1e-3, a.shape).astype(np.float32) for a in (ms, op, col)]
    v = [(rng.random(a.shape) * 1e-6).astype(np.float32) for a in (ms, op, col)]
    acc = (rng.random(n) * 4.0).astype(np.float32)
    vis = rng.integers(0, 5, n).astype(np.uint32)
    if n > 8:
        op[3] = np.nan          # kept (the comparison is false)
        acc[5] = np.nan         # never a candidate
    return (ms, op, col), m, v, acc, vis


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(p, m, v, acc, vis, sh, mode, op_min, tau_g, smin, cap):
    C = p[2].shape[1]
    scene = igs.Scene(*[_dev(a) for a in p])
    outs = [(torch.full((cap, 4), 7.0, device="cuda"), torch.full((cap,), 7.0, device="cuda"),
             torch.full((cap, C), 7.0, device="cuda")) for _ in range(3)]
    count = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    work = torch.empty(igs.densify_work_bytes(scene.n), dtype=torch.uint8, device="cuda")
    igs.densify(scene, [_dev(a) for a in m], [_dev(a) for a in v], sh, mode, _dev(acc), _dev(vis.view(np.int32)),
                op_min, tau_g, smin, outs[0], outs[1], outs[2], count, work)
    torch.cuda.synchronize()
    k = int(count.item())
    for group in outs:       # nothing written past the count
        for t in group:
            assert torch.all(t[k:] == 7.0)
    return k, [[t[:k].cpu().numpy() for t in g] for g in outs]


@pytest.mark.parametrize("n,cap", [(0, 16), (1, 8), (2047, 4000), (2049, 2049), (20011, 60000), (20011, 23000),
                                   (20011, 5000), (100003, 400000)])
@pytest.mark.parametrize("sh,mode", [(3, 1), (-1, 0)])
def test_densify_bit_exact(n, cap, sh, mode):
    C = 3 if sh < 0 else 48
    p, m, v, acc, vis = _state(n, C, 1000 + n, mode)
    op_min = 0.0 if mode == 1 else 0.3
    smin = float(np.log(0.01)) if mode == 1 else 0.01
    tau_g = 0.9
    want = oracle.densify3d(p, m, v, acc, vis, mode, op_min, tau_g, smin, cap)
    k, got = _run(p, m, v, acc, vis, sh, mode, op_min, tau_g, smin, cap)
    assert k == want[0][0].shape[0]
    for g_group, w_group in zip(got, want):
        for g, w in zip(g_group, w_group):
            np.testing.assert_array_equal(g, w.reshape(g.shape))


def test_grad_accum_bit_exact():
    rng = np.random.default_rng(8)
    n = 30001
    g = (rng.normal(size=(n, 8)) * 1e-3).astype(np.float32)
    cnt = rng.integers(0, 3, n).astype(np.uint32)
    a0 = rng.random(n).astype(np.float32)
    v0 = rng.integers(0, 9, n).astype(np.uint32)
    acc, vis = _dev(a0), _dev(v0.view(np.int32))
    igs.grad_accum(_dev(g), _dev(cnt.view(np.int32)), acc, vis)
    igs.grad_accum(_dev(g[::-1].copy()), _dev(cnt.view(np.int32)), acc, vis)
    wa, wv = oracle.grad_accum3d(g, cnt, a0, v0)
    wa, wv = oracle.grad_accum3d(g[::-1], cnt, wa, wv)
    np.testing.assert_array_equal(acc.cpu().numpy(), wa)
    np.testing.assert_array_equal(vis.cpu().numpy().view(np.uint32), wv)


def test_densify_rejects_overlap():
    p, m, v, acc, vis = _state(64, 48, 3, 1)
    scene = igs.Scene(*[_dev(a) for a in p])
    mm = [_dev(a) for a in m]
    out = (torch.empty((128, 4), device="cuda"), torch.empty(128, device="cuda"), torch.empty((128, 48), device="cuda"))
    work = torch.empty(igs.densify_work_bytes(64), dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(igs.IgsError):
        igs.densify(scene, mm, mm, 3, 1, _dev(acc), _dev(vis.view(np.int32)), 0.0, 1.0, -10.0, out, mm, out, count,
                    work)


def test_train_step_densify_matches_oracle():
    sc, cam = random_small(3000, 48, w=160, h=120, sh_degree=3, log_params=True, spread=0.8)
    target = torch.from_numpy(scenes.target_image(cam.width, cam.height, 11)).cuda()
    ts = TrainStep(torch.from_numpy(sc.means_sigma).cuda(), torch.from_numpy(sc.opacity).cuda(),
                   torch.from_numpy(sc.color).cuda(), sh_degree=3, lr=1e-2)
    ts.track_grad_norm()
    for _ in range(3):
        ts.step(cam, target, check=True)
    torch.cuda.synchronize()
    p = [t.cpu().numpy() for t in (ts.ms, ts.op, ts.col)]
    m = [t.cpu().numpy() for t in ts.m_views]
    v = [t.cpu().numpy() for t in ts.v_views]
    acc, vis = ts.accum.cpu().numpy(), ts.vis.cpu().numpy().view(np.uint32)
    assert vis.max() == 3 and (acc > 0).any()
    seen = vis > 0
    tau_g = float(np.median(acc[seen] / vis[seen]))
    want = oracle.densify3d(p, m, v, acc, vis, 1, -1.0, tau_g, float(np.log(0.02)), 6000)
    k = ts.densify(-1.0, tau_g, float(np.log(0.02)), 6000)
    assert k == want[0][0].shape[0] and k != 3000
    for got, w in zip((ts.ms, ts.op, ts.col, *ts.m_views, *ts.v_views), (*want[0], *want[1], *want[2])):
        np.testing.assert_array_equal(got.cpu().numpy(), w.reshape(tuple(got.shape)))
    assert ts.n == k and int(ts.vis.sum()) == 0
    ts.step(cam, target, check=True)          # trains on with the new set
    torch.cuda.synchronize()
    assert np.isfinite(float(ts.loss))
