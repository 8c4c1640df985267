"""Pins of the oracle's merging of 3D Gaussians (the inverse of the octant
division; Sec. 3.2, 2.5, 3.1): closed forms of small groups, the cell
assignment recomputed in numpy FP32, identities and invariances."""
import numpy as np
import pytest

import oracle

LO = (-1.0, -1.0, -1.0)


def _params(means, sigma, opac, color):
    n = len(sigma)
    ms = np.zeros((n, 4), np.float32)
    ms[:, :3] = np.asarray(means, np.float64).reshape(n, 3)
    ms[:, 3] = sigma
    return ms, np.asarray(opac, np.float32).reshape(n), np.asarray(color, np.float32).reshape(n, -1)


def _zeros(p):
    return tuple(np.zeros_like(a) for a in p)


def _merge(p, h=0.25, scale_max=1.0, param_mode=0, m=None, v=None):
    return oracle.merge3d(p, m if m is not None else _zeros(p), v if v is not None else _zeros(p), param_mode, LO, h,
                          scale_max)


def test_two_equal_weights_closed_form():
    # two Gaussians of opacity o at +-d along x in one cell: mean at the midpoint,
    # sigma^2 = s^2 + d^2 / 3, opacity 1 - (1 - o)^2, colour the midpoint colour
    d, s, o = 0.05, 0.02, 0.4
    p = _params([[0.1 - d, 0.1, 0.1], [0.1 + d, 0.1, 0.1]], [s, s], [o, o], [[1, 0, 0], [0, 0, 1]])
    (ms, op, col), (mm, mo, mc), _ = _merge(p)
    assert ms.shape == (1, 4)
    np.testing.assert_allclose(ms[0, :3], [0.1, 0.1, 0.1], rtol=0, atol=1e-7)
    assert ms[0, 3] == pytest.approx(np.sqrt(s * s + d * d / 3), rel=1e-6)
    assert op[0] == pytest.approx(1 - (1 - o) ** 2, rel=1e-6)
    np.testing.assert_allclose(col[0], [0.5, 0, 0.5], rtol=1e-6)
    assert not mm.any() and not mo.any() and not mc.any()


def test_identical_members_keep_their_shape():
    k, o = 5, 0.3
    p = _params([[0.3, -0.2, 0.55]] * k, [0.01] * k, [o] * k, [[0.2, 0.4, 0.6]] * k)
    (ms, op, col), _, _ = _merge(p)
    np.testing.assert_allclose(ms[0], [0.3, -0.2, 0.55, 0.01], rtol=1e-6)
    assert op[0] == pytest.approx(1 - (1 - o) ** k, rel=1e-6)
    np.testing.assert_allclose(col[0], [0.2, 0.4, 0.6], rtol=1e-6)


def test_opacity_capped():
    p = _params([[0.0, 0.0, 0.0]] * 4, [0.01] * 4, [0.9] * 4, [[1, 1, 1]] * 4)
    (_, op, _), _, _ = _merge(p)
    assert op[0] == np.float32(0.99)


def test_order_cells_and_eligibility_against_numpy():
    """Output = index order with each merged group at its first member's place;
    groups = equal numpy-FP32 cell indices among eligible Gaussians."""
    rng = np.random.default_rng(3)
    n = 3000
    means = rng.uniform(-1, 1.5, size=(n, 3))
    means[::97] = np.nan
    sigma = np.exp(rng.uniform(np.log(0.002), np.log(0.05), n))
    opac = rng.uniform(0.0, 0.9, n)
    opac[::53] = 0.0
    opac[::59] = 2.0 ** -61                            # below the floor: never merged
    opac[::61] = 2.0 ** -60                            # at the floor: eligible
    col = rng.uniform(0, 1, (n, 3))
    p = _params(means, sigma, opac, col)
    h, smax = 0.125, 0.02
    (ms, op, c), _, _ = _merge(p, h=h, scale_max=smax)
    inv = np.float32(1.0) / np.float32(h)
    cell = np.floor((p[0][:, :3] - np.float32(-1.0)) * inv)
    with np.errstate(invalid="ignore"):
        ok = (np.isfinite(p[0][:, :3]).all(1) & (p[0][:, 3] <= np.float32(smax)) & (p[1] >= np.float32(2.0 ** -60))
              & (cell >= 0).all(1) & (cell < 1024).all(1))
    ci = np.where(ok[:, None], cell, 0).astype(np.int64)
    key = np.where(ok, ci[:, 0] + 1024 * ci[:, 1] + 1024 * 1024 * ci[:, 2], -1)
    emitted, heads = [], {}
    for i in range(n):
        if ok[i]:
            k = key[i]
            if k in heads:
                continue
            heads[k] = i
        emitted.append(i)
    group = {k: np.nonzero(key == k)[0] for k in heads}
    assert len(ms) == len(emitted)
    for slot, i in enumerate(emitted):
        members = group.get(key[i]) if ok[i] else None
        if members is None or len(members) == 1:      # kept bit for bit
            np.testing.assert_array_equal(ms[slot].view(np.uint32), p[0][i].view(np.uint32))
            assert op[slot] == p[1][i]
        else:                                          # merged: its mean lies in the cell of the group
            assert np.all(np.floor((ms[slot, :3].astype(np.float64) + 1.0) / h) == cell[i])
    assert sum(1 for k in heads if len(group[k]) >= 2) > 50


def test_merged_moments_of_the_mixture():
    """The merged mean and scale are the mixture's first moment and its mean
    squared distance / 3, checked by sampling the mixture."""
    rng = np.random.default_rng(5)
    means = 0.3 + rng.uniform(0, 0.2, size=(6, 3))
    sigma = rng.uniform(0.005, 0.03, 6)
    opac = rng.uniform(0.2, 0.8, 6)
    p = _params(means, sigma, opac, rng.uniform(0, 1, (6, 3)))
    (ms, _, _), _, _ = _merge(p, h=1.0)
    w = opac / opac.sum()
    comp = rng.choice(6, size=2_000_000, p=w)
    x = means[comp] + rng.normal(size=(comp.size, 3)) * sigma[comp, None]
    mu = x.mean(0)
    np.testing.assert_allclose(ms[0, :3], mu, atol=3e-4)
    r2 = ((x - ms[0, :3]) ** 2).sum(1).mean()
    assert ms[0, 3] ** 2 * 3 == pytest.approx(r2, rel=5e-3)


def test_log_parameters_agree_with_linear():
    rng = np.random.default_rng(7)
    n = 400
    means = rng.uniform(-0.5, 0.5, size=(n, 3))
    sigma = np.exp(rng.uniform(np.log(0.003), np.log(0.03), n))
    opac = rng.uniform(0.05, 0.9, n)
    col = rng.normal(0, 0.3, (n, 12))
    lin = _params(means, sigma, opac, col)
    logp = _params(means, np.log(sigma), np.log(opac / (1 - opac)), col)
    (ms_l, op_l, c_l), _, _ = _merge(lin, h=0.2, scale_max=0.02)
    (ms_g, op_g, c_g), _, _ = _merge(logp, h=0.2, scale_max=np.log(0.02), param_mode=1)
    assert ms_l.shape == ms_g.shape and len(ms_l) < n
    np.testing.assert_allclose(ms_g[:, :3], ms_l[:, :3], rtol=0, atol=2e-6)
    np.testing.assert_allclose(np.exp(ms_g[:, 3].astype(np.float64)), ms_l[:, 3], rtol=2e-6)
    np.testing.assert_allclose(1 / (1 + np.exp(-op_g.astype(np.float64))), op_l, rtol=2e-6)
    np.testing.assert_allclose(c_g, c_l, rtol=1e-5, atol=1e-6)


def test_identity_and_moments_kept():
    rng = np.random.default_rng(9)
    n = 200
    p = _params(rng.uniform(-1, 1, (n, 3)), rng.uniform(0.01, 0.02, n), rng.uniform(0.1, 0.9, n),
                rng.uniform(0, 1, (n, 3)))
    m = tuple(rng.normal(size=a.shape).astype(np.float32) for a in p)
    v = tuple(rng.uniform(size=a.shape).astype(np.float32) for a in p)
    out, om, ov = _merge(p, h=0.5, scale_max=0.001, m=m, v=v)      # nothing eligible
    for a, b in zip(out + om + ov, p + m + v):
        np.testing.assert_array_equal(a, b)


def test_translation_by_whole_cells():
    rng = np.random.default_rng(11)
    n = 500
    h = 0.25
    means = rng.uniform(-0.9, 0.4, (n, 3)).astype(np.float32)
    p = _params(means, rng.uniform(0.005, 0.01, n), rng.uniform(0.1, 0.9, n), rng.uniform(0, 1, (n, 3)))
    q = (p[0].copy(), p[1], p[2])
    q[0][:, 0] += np.float32(2 * h)                     # two cells along x, exactly representable
    (a, _, _), _, _ = _merge(p, h=h)
    (b, _, _), _, _ = _merge(q, h=h)
    assert a.shape == b.shape
    np.testing.assert_allclose(b[:, 0] - a[:, 0], 2 * h, atol=2e-6)
    np.testing.assert_allclose(b[:, 1:], a[:, 1:], rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("mode", [0, 1])
def test_opacity_floor_on_the_stored_value(mode):
    """Eligibility needs opacity >= 2^-60, tested on the stored value: 2^-60
    itself, or the FP32 logit -41.58883f, merges; the next float below does not."""
    floor = np.float32(2.0 ** -60) if mode == 0 else np.float32(-41.58883)
    below = np.nextafter(floor, np.float32(-np.inf))
    for o, merges in ((floor, True), (below, False)):
        ms = np.array([[0.1, 0.1, 0.1, 0.01], [0.12, 0.1, 0.1, 0.01]], np.float32)
        if mode == 1:
            ms[:, 3] = np.log(ms[:, 3])
        op = np.array([o, 0.5 if mode == 0 else 0.0], np.float32)
        p = (ms, op, np.ones((2, 3), np.float32))
        (out, _, _), _, _ = _merge(p, scale_max=1.0, param_mode=mode)
        assert len(out) == (1 if merges else 2)


def test_small_opacities_add_up():
    # 1 - prod(1 - o_k) for opacities far below the FP64 epsilon: about sum o_k
    # (1 - o rounds to 1 there, so the product form would give 0)
    o = [1e-17, 2e-17, 3e-17]
    p = _params([[0.1, 0.1, 0.1]] * 3, [0.01] * 3, o, [[0.0, 0.5, 1.0]] * 3)
    (ms, op, col), _, _ = _merge(p)
    assert len(op) == 1 and op[0] == pytest.approx(6e-17, rel=1e-6)
    np.testing.assert_allclose(col[0], [0.0, 0.5, 1.0], rtol=1e-6)
    # the same in logits: log(o / (1 - o)) of the sum
    lp = _params([[0.1, 0.1, 0.1]] * 3, np.log([0.01] * 3), np.log(o), [[0.0, 0.5, 1.0]] * 3)
    (_, op_l, _), _, _ = _merge(lp, scale_max=0.0, param_mode=1)
    assert op_l[0] == pytest.approx(np.log(6e-17), rel=1e-6)


def test_opacity_above_one_not_merged():
    p = _params([[0.1, 0.1, 0.1]] * 3, [0.01] * 3, [1.5, 0.5, 1.0], [[1, 1, 1]] * 3)
    (ms, op, _), _, _ = _merge(p)
    assert len(op) == 2 and op[0] == np.float32(1.5)   # kept first, then the merged pair at index 1
    assert op[1] == np.float32(0.99)                    # 1 - (1 - 0.5)(1 - 1) = 1, capped
