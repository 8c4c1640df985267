"""GPU parity of the merging of 3D Gaussians (Sec. 3.2: particles merge as
well as divide; Sec. 2.5; Sec. 3.1's Octree as the pattern, so a merge undoes
an octant division) against the oracle: the count, the order and every kept
Gaussian with its moments bit for bit (both sides take the cell and eligibility
decisions on the same FP32 operations of the stored values); merged Gaussians
within bounds derived from the kernel's FP32 arithmetic (compensated sums,
means as offsets from the first member) against the oracle's FP64. Several
blocks and radix tiles with a ragged tail, RGB and SH colour, NaN, tiny,
opaque and out-of-grid inputs, empty and one-element scenes, one cell holding
almost every Gaussian."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_14244_gb300 import igs

pytestmark = pytest.mark.gpu

LO = (-1.0, -1.0, -1.0)


def _state(n, C, seed, param_mode, spread=1.0):
    rng = np.random.default_rng(seed)
    ms = np.zeros((n, 4), np.float32)
    ms[:, :3] = rng.uniform(-spread, spread, (n, 3))
    sig = np.exp(rng.uniform(np.log(0.002), np.log(0.05), n))
    ms[:, 3] = np.log(sig) if param_mode == 1 else sig
    op = (rng.normal(0, 1.5, n) if param_mode == 1 else rng.uniform(0.0, 1.0, n)).astype(np.float32)
    col = rng.normal(0, 0.3, (n, C)).astype(np.float32)
    if n > 64:
        ms[7, 0] = np.nan                          # not eligible: kept
        op[11] = np.nan                            # not eligible: kept
        ms[13, :3] = [-1.5, 0.0, 0.0]              # left of the grid: kept
        ms[17, :3] = [-1.0, -1.0, -1.0]            # exactly on the grid corner: cell (0, 0, 0)
        ms[19, :3] = [-1.0, -1.0, -1.0]
        if param_mode == 0:
            op[23] = 0.0                           # zero opacity: kept
            op[29] = 2.0 ** -61                    # below the floor: kept
            op[31] = 1.0                           # opaque: its cell's merged opacity is capped
            op[37] = 1.5                           # not an opacity: kept
        else:
            op[23] = -50.0                         # below the floor: kept
            op[29] = np.inf                        # opaque
            op[31] = 30.0                          # opaque in FP32
        op[41] = op[43] = op[47] = (2.0 ** -55 if param_mode == 0 else -38.0)   # tiny opacities, one cell
        ms[41, :3] = ms[43, :3] = ms[47, :3] = [5.01, 5.02, 5.03]   # a cell of their own, off the cloud
    m = [rng.normal(0, 1e-3, a.shape).astype(np.float32) for a in (ms, op, col)]
    v = [(rng.random(a.shape) * 1e-6 + 1e-9).astype(np.float32) for a in (ms, op, col)]
    return (ms, op, col), m, v


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(p, m, v, sh, mode, h, smax):
    n, C = p[0].shape[0], p[2].shape[1]
    scene = igs.Scene(*[_dev(a) for a in p])
    cap = max(n, 1) + 5                            # room past n: nothing may be written there
    outs = [(torch.full((cap, 4), 7.0, device="cuda"), torch.full((cap,), 7.0, device="cuda"),
             torch.full((cap, C), 7.0, device="cuda")) for _ in range(3)]
    count = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    work = torch.empty(max(igs.merge_work_bytes(n), 16), dtype=torch.uint8, device="cuda")
    igs.merge(scene, [_dev(a) for a in m], [_dev(a) for a in v], sh, mode, LO, h, smax, outs[0], outs[1], outs[2],
              count, work)
    torch.cuda.synchronize()
    k = int(count.item())
    assert 0 <= k <= n
    for group in outs:
        for t in group:
            assert torch.all(t[k:] == 7.0)
    return k, [[t[:k].cpu().numpy() for t in g] for g in outs]


U = 2.0 ** -24  # FP32 unit roundoff


def _compare(got, want, mode, h, p_in):
    """Kept rows bit for bit; merged rows (zero moments in the oracle's output,
    moments of kept rows are nonzero) within the FP32 bounds: a mean within
    32u h + 4u |mu| (offsets of at most h from the first member, compensated
    sums), a scale within 64u relative (its log within 64u + 4u |log sigma|), an
    opacity within 16u relative (its logit within 64u (1 + |logit|)), a colour
    within 16u max |c| + 4u |c| (max over the input's colours)."""
    (g_ms, g_op, g_col), g_m, g_v = got
    (w_ms, w_op, w_col), w_m, w_v = want
    assert g_ms.shape[0] == w_ms.shape[0]
    merged = ~np.any(w_m[0] != 0, axis=1) & ~np.any(w_v[0] != 0, axis=1)
    for g, w in zip(g_m + g_v, w_m + w_v):        # moments: bit for bit everywhere
        np.testing.assert_array_equal(g.reshape(w.shape), w)
    kept = ~merged
    w_col = w_col.reshape(g_col.shape)
    np.testing.assert_array_equal(g_ms[kept].view(np.uint32), w_ms[kept].view(np.uint32))
    np.testing.assert_array_equal(g_op[kept].view(np.uint32), w_op[kept].view(np.uint32))
    np.testing.assert_array_equal(g_col[kept].view(np.uint32), w_col[kept].view(np.uint32))
    gm, wm = g_ms[merged].astype(np.float64), w_ms[merged].astype(np.float64)
    assert np.all(np.isfinite(gm)) and np.all(np.isfinite(g_op[merged])) and np.all(np.isfinite(g_col[merged]))
    assert np.all(np.abs(gm[:, :3] - wm[:, :3]) <= 32 * U * h + 4 * U * np.abs(wm[:, :3]))
    go, wo = g_op[merged].astype(np.float64), w_op[merged].astype(np.float64)
    if mode == 0:
        assert np.all(np.abs(gm[:, 3] - wm[:, 3]) <= 64 * U * np.abs(wm[:, 3]))
        assert np.all(np.abs(go - wo) <= 16 * U * np.abs(wo))
    else:
        assert np.all(np.abs(gm[:, 3] - wm[:, 3]) <= 64 * U + 4 * U * np.abs(wm[:, 3]))
        assert np.all(np.abs(go - wo) <= 64 * U * (1 + np.abs(wo)))
    cmax = float(np.abs(p_in[2]).max()) if p_in[2].size else 0.0
    gc, wc = g_col[merged].astype(np.float64), w_col[merged].astype(np.float64)
    assert np.all(np.abs(gc - wc) <= 16 * U * cmax + 4 * U * np.abs(wc))
    return int(merged.sum())


@pytest.mark.parametrize("n", [0, 1, 2, 2047, 20011, 300007])
@pytest.mark.parametrize("sh,mode", [(3, 1), (-1, 0)])
def test_merge_parity(n, sh, mode):
    C = 3 if sh < 0 else 48
    p, m, v = _state(n, C, 2000 + n, mode)
    h = 0.1 if n < 100_000 else 0.04               # a few Gaussians per occupied cell
    smax = float(np.log(0.02)) if mode == 1 else 0.02
    want = oracle.merge3d(p, m, v, mode, LO, h, smax)
    k, got = _run(p, m, v, sh, mode, h, smax)
    assert k == want[0][0].shape[0]
    merged = _compare(got, want, mode, h, p)
    if n > 1000:
        assert merged > n // 100 and k < n


@pytest.mark.parametrize("mode", [0, 1])
def test_merge_one_cell_holds_everything(mode):
    # all but a few Gaussians in one cell (a long serial group), two on the grid
    # corner, three tiny ones in a cell of their own, the ineligible ones kept
    n = 5003
    p, m, v = _state(n, 3, 77, mode, spread=0.01)
    p[0][:, :3] += np.float32(0.25)                # cell (2, 2, 2) of side 0.5; the corner pair in (0, 0, 0)
    smax = 1e9
    want = oracle.merge3d(p, m, v, mode, LO, 0.5, smax)
    k, got = _run(p, m, v, -1, mode, 0.5, smax)
    assert k == want[0][0].shape[0] and k < 10
    assert _compare(got, want, mode, 0.5, p) == 3


def test_merge_far_edge_of_the_grid():
    # cells of side 3e-6 (about 25 FP32 steps near -1, so cell boundaries fall
    # between neighbouring floats): along x the cloud spans 2048 cells, so the
    # Gaussians past the grid's 1024th cell are kept; y and z within one cell
    n = 40_000
    h = 3e-6
    p, m, v = _state(n, 3, 78, 0)
    rng = np.random.default_rng(79)
    p[0][:, 0] = np.float32(-1.0) + rng.uniform(0, 2048 * h, n).astype(np.float32)
    p[0][:, 1:3] = np.float32(-1.0) + rng.uniform(0, 0.9 * h, (n, 2)).astype(np.float32)
    want = oracle.merge3d(p, m, v, 0, LO, h, 1.0)
    k, got = _run(p, m, v, -1, 0, h, 1.0)
    assert k == want[0][0].shape[0]
    merged = _compare(got, want, 0, h, p)
    assert merged > 500 and k > n // 3             # the far half kept, the near half merged


def test_merge_invalid_arguments():
    p, m, v = _state(100, 3, 1, 0)
    scene = igs.Scene(*[_dev(a) for a in p])
    outs = [(torch.zeros((100, 4), device="cuda"), torch.zeros(100, device="cuda"), torch.zeros((100, 3), device="cuda"))
            for _ in range(3)]
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    work = torch.empty(igs.merge_work_bytes(100), dtype=torch.uint8, device="cuda")
    dm, dv = [_dev(a) for a in m], [_dev(a) for a in v]
    for h in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(igs.IgsError) as e:
            igs.merge(scene, dm, dv, -1, 0, LO, h, 1.0, outs[0], outs[1], outs[2], count, work)
        assert e.value.status == igs.ERR_INVALID_ARG
    with pytest.raises(igs.IgsError):              # an output on an input
        igs.merge(scene, dm, dv, -1, 0, LO, 0.1, 1.0, (scene.means_sigma, outs[0][1], outs[0][2]), outs[1], outs[2],
                  count, work)
    with pytest.raises(igs.IgsError):
        igs.merge(scene, dm, dv, -1, 2, LO, 0.1, 1.0, outs[0], outs[1], outs[2], count, work)
    with pytest.raises(ValueError):                # outputs too small
        igs.merge(scene, dm, dv, -1, 0, LO, 0.1, 1.0, [t[:50] for t in outs[0]], outs[1], outs[2], count, work)


def test_train_step_merge_matches_oracle():
    """TrainStep.merge after a few Adam steps (moments nonzero, log parameters,
    SH degree 3): the new flat buffers hold the oracle's result, and training
    goes on with the merged set."""
    from paper_2403_14244_gb300 import scenes
    from paper_2403_14244_gb300.render import TrainStep
    from tests._tiny import random_small
    sc, cam = random_small(3000, 48, w=160, h=120, sh_degree=3, log_params=True, spread=0.8)
    target = torch.from_numpy(scenes.target_image(cam.width, cam.height, 11)).cuda()
    ts = TrainStep(torch.from_numpy(sc.means_sigma).cuda(), torch.from_numpy(sc.opacity).cuda(),
                   torch.from_numpy(sc.color).cuda(), sh_degree=3, lr=1e-2)
    for _ in range(3):
        ts.step(cam, target, check=True)
    torch.cuda.synchronize()
    p = [t.cpu().numpy() for t in (ts.ms, ts.op, ts.col)]
    m = [t.cpu().numpy() for t in ts.m_views]
    v = [t.cpu().numpy() for t in ts.v_views]
    lo, cell, smax = (-1.0, -1.0, -1.0), 0.15, float(np.log(0.05))
    want = oracle.merge3d(p, m, v, 1, lo, cell, smax)
    k = ts.merge(lo, cell, smax)
    assert k == want[0][0].shape[0] and k < 3000
    got = ((ts.ms.cpu().numpy(), ts.op.cpu().numpy(), ts.col.cpu().numpy()),
           [t.cpu().numpy() for t in ts.m_views], [t.cpu().numpy() for t in ts.v_views])
    assert _compare(got, want, 1, cell, p) > 10
    assert ts.n == k
    ts.step(cam, target, check=True)
    torch.cuda.synchronize()
    assert np.isfinite(float(ts.loss))
