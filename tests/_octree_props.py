"""Exact, vectorised properties of an Octree initialisation (Sec. 3.1: an Octree
for 3D, colour = the cell average, sigma = half the cell width) under the greedy
rule: split the splittable leaf first in the order (error descending, id
ascending; a cell's key is the smaller of its error and its parent's key) while
the non-empty leaves fit the budget. They pin the result at sizes where the
oracle's literal greedy loop is too slow:

* the Gaussians are non-empty cells in ascending cell id, and every point lies
  in exactly one of them (the leaves partition the points);
* every split cell (a strict ancestor of a leaf) precedes every splittable leaf
  in the order, and splitting the first splittable leaf would exceed the budget;
  together these fix the split set of the greedy rule;
* each Gaussian's centre, sigma, opacity and colour are those of its cell, value
  for value (the 12-bit statistics are exact integers; the error, the mean and
  the centre are recomputed with the same IEEE operations in numpy).

Only for param_mode 0 (sigma and opacity stored as they are) and RGB colours.
"""
import numpy as np


def _morton(ix, L):
    m = np.zeros(ix.shape[0], np.int64)
    for b in range(L):
        for a in range(3):
            m |= ((ix[:, a] >> b) & 1) << (3 * b + a)
    return m


def _off(l):
    return ((1 << (3 * l)) - 1) // 7


def check_octree(p, c, lo, side, L, k_max, ms, op, col, opacity):
    """Assert the properties above for points p [n, 3], colours c [n, 3] (float32,
    all finite) and the Gaussians (ms [K, 4], op [K], col [K, 3]) made from them."""
    f32 = np.float32
    K = ms.shape[0]
    assert 1 <= K <= k_max
    # finest cell of every point: FP32 steps, each rounded once, clamped into the cube
    inv = f32(float(1 << L) / float(side))
    ix = np.empty((p.shape[0], 3), np.int64)
    for a in range(3):
        t = np.floor((p[:, a] - f32(lo[a])) * inv)
        ix[:, a] = np.clip(t, 0, (1 << L) - 1).astype(np.int64)
    mL = _morton(ix, L)
    q = np.rint(np.clip(c, 0, 1).astype(f32) * f32(4096)).astype(np.int64)
    # exact statistics and keys, level by level (float64 bincounts of integers below 2^53 are exact)
    n, s1, s2, key, m_of = [], [], [], [], []
    for l in range(L + 1):
        m = mL >> (3 * (L - l))
        m_of.append(m)
        cells = 1 << (3 * l)
        n.append(np.bincount(m, minlength=cells).astype(np.int64))
        s1.append(np.stack([np.rint(np.bincount(m, weights=q[:, ch].astype(np.float64), minlength=cells))
                            for ch in range(3)], 1).astype(np.int64))
        s2.append(np.stack([np.rint(np.bincount(m, weights=(q[:, ch] ** 2).astype(np.float64), minlength=cells))
                            for ch in range(3)], 1).astype(np.int64))
        nn = np.maximum(n[l], 1).astype(np.float64)
        e = np.zeros(cells)
        for ch in range(3):
            a1 = s1[l][:, ch].astype(np.float64)
            e = e + (s2[l][:, ch].astype(np.float64) - (a1 * a1) / nn)
        e = np.where((n[l] > 0) & (e > 0), e, 0.0)
        key.append(e if l == 0 else np.minimum(e, key[l - 1][np.arange(cells) >> 3]))
    # flat arrays over all cells, by cell id
    n_all, s1_all, key_all = np.concatenate(n), np.concatenate(s1), np.concatenate(key)
    # the Gaussians' cells
    level_of = {float(f32(0.5 * float(side) / float(1 << l))): l for l in range(L + 1)}
    lv = np.array([level_of.get(h, -1) for h in ms[:, 3].tolist()], np.int64)
    assert np.all(lv >= 0), "sigma is not half of a cell side"
    cs = float(side) / (1 << lv).astype(np.float64)
    c3 = np.rint((ms[:, :3].astype(np.float64) - np.asarray(lo, np.float64)) / cs[:, None] - 0.5).astype(np.int64)
    assert np.all(c3 >= 0) and np.all(c3 < (1 << lv)[:, None])
    mor = np.zeros(K, np.int64)
    for b in range(L):
        for a in range(3):
            mor |= np.where(b < lv, ((c3[:, a] >> b) & 1) << (3 * b + a), 0)
    offs = np.array([_off(l) for l in range(L + 2)], np.int64)
    ids = offs[lv] + mor
    assert np.all(np.diff(ids) > 0), "not in ascending cell id"
    # values of each Gaussian from its cell
    want_xyz = (np.asarray(lo, np.float64)[None, :] + (c3 + 0.5) * cs[:, None]).astype(f32)
    np.testing.assert_array_equal(ms[:, :3], want_xyz)
    np.testing.assert_array_equal(op, np.full(K, f32(opacity)))
    n_leaf = n_all[ids]
    assert np.all(n_leaf > 0), "an empty cell holds a Gaussian"
    want_col = (s1_all[ids].astype(np.float64) / (4096.0 * n_leaf.astype(np.float64))[:, None]).astype(f32)
    np.testing.assert_array_equal(col, want_col)
    # the leaves partition the points
    leaf = [np.zeros(1 << (3 * l), bool) for l in range(L + 1)]
    for l in range(L + 1):
        leaf[l][mor[lv == l]] = True
    hits = np.zeros(p.shape[0], np.int64)
    for l in range(L + 1):
        hits += leaf[l][m_of[l]]
    assert np.all(hits == 1), "the leaves do not partition the points"
    # split cells: non-empty, not a leaf, not below a leaf
    below = np.zeros(1, bool)
    s_key, s_id = [], []
    for l in range(L + 1):
        cells = 1 << (3 * l)
        if l > 0:
            below = (below | leaf[l - 1])[np.arange(cells) >> 3]
        split = (n[l] > 0) & ~leaf[l] & ~below
        assert not (l == L and split.any())
        s_key.append(key[l][split])
        s_id.append(_off(l) + np.flatnonzero(split))
    s_key, s_id = np.concatenate(s_key), np.concatenate(s_id)
    # splittable leaves: >= 2 points above the finest level; what a split would add
    u = (lv < L) & (n_leaf >= 2)
    u_key, u_id = key_all[ids[u]], ids[u]
    kids = offs[lv[u] + 1][:, None] + 8 * mor[u][:, None] + np.arange(8)[None, :]
    u_inc = (n_all[kids] > 0).sum(1) - 1
    if s_key.size and u_key.size:
        # the last split cell in the order precedes the first splittable leaf
        ls = np.lexsort((-s_id, s_key))[0]            # smallest key, then largest id
        fu = np.lexsort((u_id, -u_key))[0]            # largest key, then smallest id
        assert s_key[ls] > u_key[fu] or (s_key[ls] == u_key[fu] and s_id[ls] < u_id[fu]), \
            "a splittable leaf precedes a split cell in the order"
    if u_key.size:
        fu = np.lexsort((u_id, -u_key))[0]
        assert K + u_inc[fu] > k_max, "the next split of the order still fits the budget"
