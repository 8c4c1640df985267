"""GPU parity of the adjoint (backward blend + projection backward) against
the oracle's FP64 analytic gradients (themselves pinned by finite differences
and torch autograd), and of the L1 loss and Adam kernels."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2403_14244_gb300 import igs, scenes
from paper_2403_14244_gb300.render import TrainStep
from tests import _gpu
from tests._tiny import random_small, scene_from, small_camera

pytestmark = pytest.mark.gpu


def _gpu_grads(sc, cam, W, tile=16, bg=(0.0, 0.0, 0.0), footprint=0):
    r, f, scene, img = _gpu.run_forward(sc, cam, tile=tile, bg=bg, footprint=footprint)
    dimg = torch.from_numpy(np.ascontiguousarray(W, np.float32)).cuda()
    d_ms, d_op, d_col = r.run_backward(scene, cam, f, dimg)
    torch.cuda.synchronize()
    return img, d_ms.cpu().numpy(), d_op.cpu().numpy(), d_col.cpu().numpy()


def _compare(sc, cam, W, tile=16, bg=(0.0, 0.0, 0.0), footprint=0, **tol):
    img, d_ms, d_op, d_col = _gpu_grads(sc, cam, W, tile, bg, footprint)
    ref = oracle.backward(sc, cam, W, mode=1, bg=bg)
    out = {}
    out["means"] = _gpu.grad_close(d_ms[:, :3], ref["d_means"], "means", **tol)
    out["sigma"] = _gpu.grad_close(d_ms[:, 3], ref["d_sigma"], "sigma", **tol)
    out["opacity"] = _gpu.grad_close(d_op, ref["d_opac"], "opacity", **tol)
    out["color"] = _gpu.grad_close(d_col, ref["d_color"], "color", **tol)
    return out, ref


@pytest.mark.parametrize("footprint", [0, 1])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_backward_rgb_small(tile, footprint):
    sc, cam = random_small(300, 41, w=80, h=60, spread=0.8)
    W = np.random.default_rng(1).normal(size=(3, cam.height, cam.width))
    _compare(sc, cam, W, tile=tile, footprint=footprint)


def test_backward_sh3_log_background():
    sc, cam = random_small(300, 42, w=80, h=60, sh_degree=3, log_params=True, spread=0.8)
    W = np.random.default_rng(2).normal(size=(3, cam.height, cam.width))
    _compare(sc, cam, W, bg=(0.25, 0.5, 0.125))


def test_backward_clamp_active():
    sc, cam = random_small(200, 43, w=64, h=48, spread=0.6)
    sc.opacity[::3] = np.float32(0.999)
    W = np.random.default_rng(3).normal(size=(3, cam.height, cam.width))
    _compare(sc, cam, W)


def test_backward_clustered_1080p_full():
    """Full 1M-Gaussian SH3 1080p case with the L1 gradient of a seeded target;
    every Gaussian in norm, and a 64-Gaussian subset (seed 202, among those that
    were blended somewhere) element by element."""
    sc, cam, target = scenes.workload_fwd_bwd_1m()
    r, f, scene, img = _gpu.run_forward(sc, cam)
    ref_fwd = oracle.render(sc, cam, mode=1)
    # the same dL/dimg on both sides: the oracle's L1 gradient of its own image
    _, G = oracle.l1(ref_fwd["img"], target)
    img_gpu, d_ms, d_op, d_col = _gpu_grads(sc, cam, G)
    ref = oracle.backward(sc, cam, G, mode=1)
    _gpu.grad_close(d_ms[:, :3], ref["d_means"], "means")
    _gpu.grad_close(d_ms[:, 3], ref["d_sigma"], "sigma")
    _gpu.grad_close(d_op, ref["d_opac"], "opacity")
    _gpu.grad_close(d_col, ref["d_color"], "color")
    hit = np.nonzero(np.abs(ref["g2d"]).sum(axis=1) > 0)[0]
    sub = np.random.default_rng(202).choice(hit, size=64, replace=False)
    for name, g, w in (("means", d_ms[sub, :3], ref["d_means"][sub]), ("sigma", d_ms[sub, 3], ref["d_sigma"][sub]),
                       ("opacity", d_op[sub], ref["d_opac"][sub]), ("color", d_col[sub], ref["d_color"][sub])):
        _gpu.grad_close(g, w, name + "[subset]", rel_norm=1e-3, elem_rel=1e-3, elem_abs_frac=1e-3)


@pytest.mark.parametrize("shape", [(3, 70, 90), (3, 7, 5)])   # float4 path; a count not a multiple of 4
def test_l1_loss_matches_oracle(shape):
    rng = np.random.default_rng(5)
    img = rng.uniform(size=shape).astype(np.float32)
    tg = rng.uniform(size=shape).astype(np.float32)
    tg[0, :5, :5] = img[0, :5, :5]
    ti, tt = torch.from_numpy(img).cuda(), torch.from_numpy(tg).cuda()
    loss = torch.zeros(1, device="cuda")
    grad = torch.empty_like(ti)
    igs.l1_loss(ti, tt, loss, grad)
    want, g_ref = oracle.l1(img.astype(np.float64), tg)
    assert float(loss) == pytest.approx(want, rel=1e-5)
    np.testing.assert_allclose(grad.cpu().numpy(), g_ref, rtol=1e-6)


def test_adam_matches_oracle():
    rng = np.random.default_rng(6)
    n = 10_001                                                   # odd: vector body plus scalar tail
    p0 = rng.normal(size=n).astype(np.float32)
    p, m, v = (torch.from_numpy(p0).cuda(), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda"))
    rp, rm, rv = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 6):
        g = (rng.normal(size=n) * (0.01 if t % 2 else 3.0)).astype(np.float32)
        igs.adam(p, torch.from_numpy(g).cuda(), m, v, t, lr=1e-3)
        rp, rm, rv = oracle.adam(rp, g, rm, rv, lr=1e-3, t=t)
    np.testing.assert_allclose(p.cpu().numpy(), rp, rtol=0, atol=2e-6)
    # m mixes terms of size (1 - b1) |g| <= 0.3 whose sum can cancel: a few FP32 ulp of 0.3
    np.testing.assert_allclose(m.cpu().numpy(), rm, rtol=1e-5, atol=4 * np.spacing(np.float32(0.3)))
    np.testing.assert_allclose(v.cpu().numpy(), rv, rtol=1e-5, atol=1e-12)


def _flat_ref(sc, ref):
    return (np.concatenate([ref["d_means"], ref["d_sigma"][:, None]], 1), ref["d_opac"], ref["d_color"])


def test_train_step_matches_oracle():
    """One full step (forward, L1, backward, Adam) on a log-parameter SH3 scene,
    unfused (gradient written, then Adam) and fused (projection backward + Adam)."""
    sc, cam = random_small(500, 44, w=96, h=64, sh_degree=3, log_params=True, spread=0.8)
    target = scenes.target_image(cam.width, cam.height, 9)
    ref_fwd = oracle.render(sc, cam, mode=1)
    loss_ref, G = oracle.l1(ref_fwd["img"], target)
    ref = oracle.backward(sc, cam, G, mode=1)
    g_ms, g_op, g_col = _flat_ref(sc, ref)
    outs = {}
    for fused in (False, True):
        ts = TrainStep(torch.from_numpy(sc.means_sigma).cuda(), torch.from_numpy(sc.opacity).cuda(),
                       torch.from_numpy(sc.color).cuda(), sh_degree=3, lr=1e-3, fused=fused)
        ts.step(cam, torch.from_numpy(target).cuda(), check=True)
        torch.cuda.synchronize()
        assert float(ts.loss) == pytest.approx(loss_ref, rel=1e-4)
        if not fused:
            _gpu.grad_close(ts.g_ms.cpu().numpy(), g_ms, "means_sigma grad")
            _gpu.grad_close(ts.g_op.cpu().numpy(), g_op, "opacity grad")
            _gpu.grad_close(ts.g_col.cpu().numpy(), g_col, "color grad")
        outs[fused] = [t.cpu().numpy() for t in (ts.ms, ts.op, ts.col, *ts.m_views, *ts.v_views)]
        for name, p0, g, got in (("means_sigma", sc.means_sigma, g_ms, outs[fused][0]),
                                 ("opacity", sc.opacity, g_op, outs[fused][1]),
                                 ("color", sc.color, g_col, outs[fused][2])):
            p_ref, _, _ = oracle.adam(p0.astype(np.float64), g, np.zeros(g.shape), np.zeros(g.shape), lr=1e-3, t=1)
            # first Adam step moves a parameter with a non-tiny gradient by ~lr * sign(g)
            moved = np.abs(g) > 1e-3 * np.abs(g).max()
            np.testing.assert_allclose(got[moved], p_ref[moved], atol=2e-6, err_msg=name)
            still = g == 0
            np.testing.assert_array_equal(got[still], p0[still])
    # fused and unfused steps agree (same FP32 arithmetic up to the gradient's summation order)
    for a, b in zip(outs[False], outs[True]):
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-7)


def test_fused_adam_ragged_and_repeated():
    """Fused projection backward + Adam on a scene whose size is not a multiple of
    the 32-Gaussian warp tile, over three steps, against the unfused path."""
    sc, cam = random_small(1001, 45, w=80, h=60, sh_degree=3, log_params=True, spread=0.8)
    target = torch.from_numpy(scenes.target_image(cam.width, cam.height, 10)).cuda()
    states = []
    for fused in (False, True):
        ts = TrainStep(torch.from_numpy(sc.means_sigma).cuda(), torch.from_numpy(sc.opacity).cuda(),
                       torch.from_numpy(sc.color).cuda(), sh_degree=3, lr=1e-2, fused=fused)
        for _ in range(3):
            ts.step(cam, target, check=True)
        torch.cuda.synchronize()
        states.append(torch.cat([ts.flat, ts.m, ts.v]).cpu().numpy())
    np.testing.assert_allclose(states[0], states[1], rtol=1e-4, atol=1e-6)


def test_train_step_graph_replay_matches_eager():
    """Training steps replayed from CUDA graphs (one per view, the Adam step
    count on the device) follow the same trajectory as eager steps: same
    parameters and moments up to the backward's atomic summation order, and the
    device step count advances once per replay."""
    sc, cam = random_small(2000, 49, w=128, h=96, sh_degree=3, log_params=True, spread=0.8)
    cams = [cam, dataclasses.replace(cam, t=(np.asarray(cam.t, np.float32) + np.float32(0.05)).astype(np.float32))]
    targets = [torch.from_numpy(scenes.target_image(cam.width, cam.height, 20 + k)).cuda() for k in range(2)]
    states = []
    for graphed in (False, True):
        ts = TrainStep(torch.from_numpy(sc.means_sigma).cuda(), torch.from_numpy(sc.opacity).cuda(),
                       torch.from_numpy(sc.color).cuda(), sh_degree=3, lr=1e-2)
        for k in range(2):  # capacity calibration (also the first two steps)
            ts.step(cams[k], targets[k], check=True)
        if graphed:
            ts.capture(cams, targets)
            for k in range(6):
                ts.replay(k % 2)
        else:
            for k in range(6):
                ts.step(cams[k % 2], targets[k % 2])
        torch.cuda.synchronize()
        assert int(ts.adam_state[0]) == 8
        states.append(torch.cat([ts.flat, ts.m, ts.v]).cpu().numpy())
    np.testing.assert_allclose(states[0], states[1], rtol=1e-4, atol=1e-6)


def test_train_step_full_size_graph_replay():
    """The benchmark's training step at full size and in its launch configuration: 3M SH3 Gaussians
    (log sigma, logit opacity), view 5 at 1297x840, 32-pixel tiles, projection backward and Adam
    fused, replayed from a CUDA graph, from a clean Adam state (t = 1). The L1 target is the
    oracle's own image plus a seeded +-0.25 per entry, so the sign of the L1 gradient is the same
    on both sides wherever the images agree to 0.25. Checked: the loss; the gradient, read from the
    first moment (m = (1 - beta1) g at t = 1), against the oracle's in norm over all 3M Gaussians and
    element by element on 64 of those that were blended; the updated parameters against the
    oracle's Adam step wherever the gradient is not tiny, and unchanged where the step's gradient is
    zero."""
    sc, cams = scenes.workload_train_3m()
    cam = cams[5]
    ref_fwd = oracle.render(sc, cam, mode=1)
    sign = np.random.default_rng(505).choice([-1.0, 1.0], size=ref_fwd["img"].shape)
    target = (ref_fwd["img"] + 0.25 * sign).astype(np.float32)
    loss_ref, G = oracle.l1(ref_fwd["img"], target)
    ts = TrainStep(torch.from_numpy(sc.means_sigma).cuda(), torch.from_numpy(sc.opacity).cuda(),
                   torch.from_numpy(sc.color).cuda(), sh_degree=3, tile=32, lr=1e-3)
    tgt = torch.from_numpy(target).cuda()
    c = igs.camera(cam)
    ts.step(c, tgt, check=True)  # entry capacity of the view (also one step)
    ts.capture([c], [tgt])
    # back to the initial state: parameters, moments and the device step count
    ts.ms.copy_(torch.from_numpy(sc.means_sigma))
    ts.op.copy_(torch.from_numpy(sc.opacity))
    ts.col.copy_(torch.from_numpy(sc.color))
    ts.m.zero_()
    ts.v.zero_()
    ts.adam_state.zero_()
    ts.replay(0)
    torch.cuda.synchronize()
    assert int(ts.adam_state[0]) == 1
    assert float(ts.loss) == pytest.approx(loss_ref, rel=1e-4)
    ref = oracle.backward(sc, cam, G, mode=1)
    want = _flat_ref(sc, ref)
    got = [m.cpu().numpy().astype(np.float64) / np.float64(np.float32(0.1)) for m in ts.m_views]
    hit = np.nonzero(np.abs(ref["g2d"]).sum(axis=1) > 0)[0]
    sub = np.random.default_rng(606).choice(hit, size=64, replace=False)
    for name, g, w in zip(("means_sigma", "opacity", "color"), got, want):
        _gpu.grad_close(g, w, name)
        _gpu.grad_close(g[sub], w[sub], name + "[subset]", rel_norm=1e-3, elem_rel=1e-3, elem_abs_frac=1e-3)
    for name, p0, w, g, p in (("means_sigma", sc.means_sigma, want[0], got[0], ts.ms),
                              ("opacity", sc.opacity, want[1], got[1], ts.op), ("color", sc.color, want[2], got[2], ts.col)):
        p = p.cpu().numpy()
        p_ref, _, _ = oracle.adam(p0.astype(np.float64), w, np.zeros(w.shape), np.zeros(w.shape), lr=1e-3, t=1)
        moved = np.abs(w) > 1e-2 * np.abs(w).max()
        assert moved.sum() > 100, name
        np.testing.assert_allclose(p[moved], p_ref[moved], atol=2e-6, err_msg=name)
        np.testing.assert_array_equal(p[g == 0], p0[g == 0])


def _frame_arrays(f, footprint):
    out = [f.rec(), f.rect(), f.count(), f.depth_key()] + ([f.disc()] if footprint else [])
    return [a.cpu().numpy().view(np.uint32) for a in out]


@pytest.mark.parametrize("sh,footprint", [(3, 0), (3, 1), (-1, 0), (1, 1)])
def test_fused_next_projection_bit_exact(sh, footprint):
    """A step with next_cam projects the updated scene for the next view in its
    last pass: the frame then holds exactly what a separate projection of the
    updated parameters writes (same size: in the step's own frame; another
    size: in that size's frame), for staged (SH 3, 1) and unstaged (RGB) colour
    rows, both footprints, a ragged last warp of Gaussians."""
    C = 3 if sh < 0 else 3 * (sh + 1) ** 2
    sc, cam = random_small(1001, 46, w=96, h=64, sh_degree=sh, log_params=True, spread=0.8)
    cam2 = dataclasses.replace(cam, t=(np.asarray(cam.t, np.float32) + np.float32(0.07)).astype(np.float32))
    cam3 = dataclasses.replace(cam2, width=80, height=72, cx=40.0, cy=36.0)
    target = torch.from_numpy(scenes.target_image(cam.width, cam.height, 12)).cuda()
    ts = TrainStep(torch.from_numpy(sc.means_sigma).cuda(), torch.from_numpy(sc.opacity).cuda(),
                   torch.from_numpy(sc.color.reshape(sc.n, C)).cuda(), sh_degree=sh, lr=1e-2, footprint=footprint)
    for nxt in (cam2, cam3):
        ts.step(cam, target, check=True)           # capacity of the view
        ts.step(igs.camera(nxt), torch.zeros((3, nxt.height, nxt.width), device="cuda"), check=True)
        ts.step(cam, target, next_cam=nxt)
        torch.cuda.synchronize()
        r = ts.renderer
        c = igs.camera(nxt)
        f_fused = r.frame(ts.n, c, r.capacity_for(ts.n, c))
        got = _frame_arrays(f_fused, footprint)
        ref = igs.Frame(ts.n, 1 << 16, c, r.opts)
        igs.project(ts.scene, c, r.opts, ref)
        torch.cuda.synchronize()
        for g, w in zip(got, _frame_arrays(ref, footprint)):
            np.testing.assert_array_equal(g, w)
        assert (got[2] > 0).sum() > 500


def test_chained_steps_and_graphs_match_plain_steps():
    """Steps that project the next view in their last pass (eager, and replayed
    from chained CUDA graphs in order and out of order) follow the trajectory of
    plain steps: parameters and moments agree up to the backward's atomic
    summation order, and the device step count advances once per step."""
    sc, cam = random_small(2000, 49, w=128, h=96, sh_degree=3, log_params=True, spread=0.8)
    cams = [igs.camera(dataclasses.replace(cam, t=(np.asarray(cam.t, np.float32) + np.float32(0.04 * k))
                                           .astype(np.float32))) for k in range(3)]
    targets = [torch.from_numpy(scenes.target_image(cam.width, cam.height, 30 + k)).cuda() for k in range(3)]
    order = [0, 1, 2, 0, 1, 2, 2, 1, 0, 1]            # in order, then out of order
    states = []
    for mode in ("plain", "chained", "graphs"):
        ts = TrainStep(torch.from_numpy(sc.means_sigma).cuda(), torch.from_numpy(sc.opacity).cuda(),
                       torch.from_numpy(sc.color).cuda(), sh_degree=3, lr=1e-2)
        for k in range(3):
            ts.step(cams[k], targets[k], check=True)
        if mode == "graphs":
            ts.capture(cams, targets, chain=True)
            for k in order:
                ts.replay(k)
        else:
            for j, k in enumerate(order):
                nxt = cams[order[j + 1]] if mode == "chained" and j + 1 < len(order) else None
                ts.step(cams[k], targets[k], next_cam=nxt)
        torch.cuda.synchronize()
        assert int(ts.adam_state[0]) == 3 + len(order)
        states.append(torch.cat([ts.flat, ts.m, ts.v]).cpu().numpy())
    np.testing.assert_allclose(states[1], states[0], rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(states[2], states[0], rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("tile", [16, 32])
def test_backward_long_walks_cut_into_segments(tile):
    """Many faint, wide Gaussians over a small image: no pixel saturates, so each
    8 x 8 block walks thousands of its tile's entries and the forward cuts the
    walks into segments of 1024 list positions, which the backward walks in
    parallel from the saved states. The gradients match the oracle's as a single
    reverse walk's do; the image is unaffected."""
    rng = np.random.default_rng(47)
    n = 5000
    cam = small_camera(64, 48, 80.0)
    means = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.45, 0.45, n), rng.uniform(-0.5, 0.5, n)], 1)
    # opacity 0.0042-0.006: only the core of each disc blends (alpha >= 1/255), a
    # few hundred Gaussians per pixel, and no pixel reaches t_min
    sc = scene_from(means, rng.uniform(0.3, 0.6, n), rng.uniform(0.0042, 0.006, n), rng.uniform(0, 1, (n, 3)))
    W = rng.normal(size=(3, cam.height, cam.width))
    r, f, scene, img = _gpu.run_forward(sc, cam, tile=tile)
    assert igs.frame_walk_segments(f) > 20            # the walks were cut
    ref = oracle.render(sc, cam, mode=1, flag_margin=1e-5)
    assert ref["T"].min() > 2e-4 and ref["last"].max() > 4000   # no pixel stops; walks of ~5000 entries
    # opacities this close to 1/255 put some 2 % of pixels within the oracle's
    # margin of an alpha_min decision (flagged, left out of the comparison)
    _gpu.compare_images(img, ref["img"], ref["flag"], atol=2e-4, max_flag_frac=0.03)
    _compare(sc, cam, W, tile=tile)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_forward_clear_then_accumulating_backward(tile):
    """igs_render_fwd_clear + igs_blend_bwd_acc (the training step's pair: the
    forward's CTAs zero g2d, the backward accumulates without a clearing pass)
    give the image of igs_render_fwd bit for bit and the screen-space gradients
    of igs_render_fwd + igs_blend_bwd, starting from a g2d full of garbage; the
    backward's work counter is reset by the forward, so the pair repeats on one
    frame. An aborted frame (capacity) still leaves g2d cleared."""
    sc, cam = random_small(3000, 48, w=160, h=96, spread=0.8)
    W = np.random.default_rng(5).normal(size=(3, cam.height, cam.width))
    dimg = torch.from_numpy(np.ascontiguousarray(W, np.float32)).cuda()
    r, f, scene, img = _gpu.run_forward(sc, cam, tile=tile)
    o = r.opts
    g_ref = torch.full((sc.n, 8), 7.0, device="cuda")
    igs.blend_bwd(f, o, dimg, g_ref)
    img_ref = torch.from_numpy(img.astype(np.float32)).cuda()   # the GPU image, back from float64 exactly
    for _ in range(2):
        g = torch.full((sc.n, 8), float("nan"), device="cuda")
        out = torch.full_like(img_ref, -1.0)
        igs.render_fwd_clear(f, o, out, g)
        igs.blend_bwd_acc(f, o, dimg, g)
        torch.cuda.synchronize()
        assert torch.equal(out, img_ref)
        a, b = g.cpu().numpy().astype(np.float64), g_ref.cpu().numpy().astype(np.float64)
        assert np.isfinite(a).all()
        # float atomics add in a different order from run to run: a few ulp
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())
    # capacity overflow: nothing is blended, g2d is still cleared
    c = igs.camera(cam)
    small = igs.Frame(scene.n, 16, c, o)
    igs.project(scene, c, o, small)
    igs.bin_sort(small, o)
    g = torch.full((sc.n, 8), 3.0, device="cuda")
    igs.render_fwd_clear(small, o, torch.zeros_like(img_ref), g)
    igs.blend_bwd_acc(small, o, dimg, g)
    st, _ = igs.frame_status(small)
    assert st == igs.ERR_CAPACITY
    assert torch.count_nonzero(g).item() == 0


def test_forward_clear_binding_refuses_small_g2d():
    sc, cam = random_small(50, 49, w=32, h=32)
    r, f, scene, img = _gpu.run_forward(sc, cam, tile=16)
    out = torch.zeros((3, 32, 32), device="cuda")
    with pytest.raises(ValueError):
        igs.render_fwd_clear(f, r.opts, out, torch.zeros((sc.n - 1, 8), device="cuda"))
    with pytest.raises(ValueError):
        igs.blend_bwd_acc(f, r.opts, out, torch.zeros((sc.n, 8), device="cuda", dtype=torch.float64))


def test_graphs_with_host_copies_match_device_targets():
    """Steps whose graphs copy the target in from pinned host memory and the loss
    out to it (TrainStep.capture with targets_host / losses_host) follow the
    trajectory of graphs that read targets already on the device, and each
    view's host loss is that step's loss. The device target buffers start as
    garbage, so a step that read them before its copy landed would diverge."""
    sc, cam = random_small(2000, 51, w=128, h=96, sh_degree=3, log_params=True, spread=0.8)
    cams = [igs.camera(dataclasses.replace(cam, t=(np.asarray(cam.t, np.float32) + np.float32(0.04 * k))
                                           .astype(np.float32))) for k in range(3)]
    host = [torch.from_numpy(scenes.target_image(cam.width, cam.height, 40 + k)).pin_memory() for k in range(3)]
    order = [0, 1, 2, 0, 1, 2, 0]
    states, losses = [], []
    for mode in ("device", "host"):
        ts = TrainStep(torch.from_numpy(sc.means_sigma).cuda(), torch.from_numpy(sc.opacity).cuda(),
                       torch.from_numpy(sc.color).cuda(), sh_degree=3, lr=1e-2)
        targets = [t.cuda() for t in host]
        for k in range(3):
            ts.step(cams[k], targets[k], check=True)
        if mode == "device":
            ts.capture(cams, targets, chain=True)
            got = []
            for k in order:
                ts.replay(k)
                got.append(ts.loss.clone())
        else:
            lh = [torch.full((1,), float("nan")).pin_memory() for _ in range(3)]
            ts.capture(cams, targets, chain=True, targets_host=host, losses_host=lh)
            for t in targets:
                t.fill_(-5.0)                       # the graphs must copy the real targets in
            got = []
            for k in order:
                ts.replay(k)
                torch.cuda.synchronize()
                assert float(lh[k]) == float(ts.loss)
                got.append(lh[k].clone())
        torch.cuda.synchronize()
        states.append(torch.cat([ts.flat, ts.m, ts.v]).cpu().numpy())
        losses.append([float(x) for x in got])
    np.testing.assert_allclose(states[1], states[0], rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(losses[1], losses[0], rtol=1e-5)


def test_checkpoint_resume_matches_uninterrupted(tmp_path):
    """Training state saved after some steps (parameters, Adam moments, step
    count, densify statistic) and loaded into a new TrainStep continues as the
    uninterrupted run does: same parameters and moments after five more steps,
    up to the backward's atomic summation order, and the same step count."""
    sc, cam = random_small(2000, 52, w=128, h=96, sh_degree=3, log_params=True, spread=0.8)
    cams = [igs.camera(dataclasses.replace(cam, t=(np.asarray(cam.t, np.float32) + np.float32(0.04 * k))
                                           .astype(np.float32))) for k in range(3)]
    targets = [torch.from_numpy(scenes.target_image(cam.width, cam.height, 60 + k)).cuda() for k in range(3)]
    ts = TrainStep(torch.from_numpy(sc.means_sigma).cuda(), torch.from_numpy(sc.opacity).cuda(),
                   torch.from_numpy(sc.color).cuda(), sh_degree=3, lr=1e-2)
    ts.track_grad_norm()
    for k in (0, 1, 2, 0):
        ts.step(cams[k], targets[k], check=True)
    path = tmp_path / "train_state.pt"
    ts.save(path)
    after = (1, 2, 0, 1, 2)
    for k in after:
        ts.step(cams[k], targets[k], check=True)
    ts2 = TrainStep.load(path)
    assert ts2.t == 4 and ts2.accum is not None
    for k in after:
        ts2.step(cams[k], targets[k], check=True)
    torch.cuda.synchronize()
    assert ts2.t == ts.t and torch.equal(ts2.adam_state[:1], ts.adam_state[:1])
    a = torch.cat([ts.flat, ts.m, ts.v]).cpu().numpy()
    b = torch.cat([ts2.flat, ts2.m, ts2.v]).cpu().numpy()
    np.testing.assert_allclose(b, a, rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(ts2.accum.cpu().numpy(), ts.accum.cpu().numpy(), rtol=1e-4, atol=1e-9)
    np.testing.assert_array_equal(ts2.vis.cpu().numpy(), ts.vis.cpu().numpy())


@pytest.mark.parametrize("fused", [False, True])
def test_projection_backward_ignores_culled_rows_of_g2d(fused):
    """The projection backward loads every Gaussian's row of the 2D gradient
    together with its other values, but uses only the rows of Gaussians that
    touch a tile: NaN in the rows of culled Gaussians changes no output bit,
    in the plain projection backward and in the one fused with Adam (whose
    culled Gaussians take a zero gradient)."""
    sc, cam = random_small(600, 48, w=80, h=60, sh_degree=3, log_params=True, spread=1.6)
    r, f, scene, _ = _gpu.run_forward(sc, cam, tile=16)
    c = igs.camera(cam)
    n = scene.n
    culled = f.count() == 0
    assert 0 < int(culled.sum()) < n
    dimg = torch.from_numpy(np.random.default_rng(5).normal(size=(3, cam.height, cam.width)).astype(np.float32)).cuda()
    g2d = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    igs.blend_bwd(f, r.opts, dimg, g2d)
    g_nan = g2d.clone()
    g_nan[culled] = float("nan")
    outs = []
    for g in (g2d, g_nan):
        if not fused:
            ts = (torch.empty_like(scene.means_sigma), torch.empty_like(scene.opacity), torch.empty_like(scene.color))
            igs.project_bwd(scene, c, r.opts, f, g, *ts)
        else:
            s2 = igs.Scene(scene.means_sigma.clone(), scene.opacity.clone(), scene.color.clone())
            m = [torch.zeros_like(t) for t in (s2.means_sigma, s2.opacity, s2.color)]
            v = [torch.zeros_like(t) for t in (s2.means_sigma, s2.opacity, s2.color)]
            igs.project_bwd_adam(s2, c, r.opts, f, g, m, v, step=1, lr=1e-2)
            ts = (s2.means_sigma, s2.opacity, s2.color, *m, *v)
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in ts])
    for a, b in zip(*outs):
        assert np.isfinite(a).all()
        np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
