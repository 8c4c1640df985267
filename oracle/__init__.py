"""CPU oracle for isotropic Gaussian splatting (arXiv 2403.14244).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark are the only callers. The product path never imports this
package, and this package imports nothing from the product path except the
seeded input generators (``paper_2403_14244_gb300.scenes``), which hold none of
the method's arithmetic.

The arithmetic lives in ``igs_oracle.c`` (plain C, FP64 compositing and
gradients, canonical FP32 key path), built here with gcc and loaded with
ctypes. Every function states the passage of the paper it follows; the readings
taken where the paper is silent are listed at the top of ``igs_oracle.c``.

Parity pins: every function here is checked by the ``-m "not gpu"`` tests
against closed forms, brute force, invariants, finite differences, scipy's
spherical harmonics and Gaussian filter, and torch's Adam / L1 / conv2d autograd
(see tests/test_oracle_*.py).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "igs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
          "-fPIC", "-shared", "-Wall", "-Wno-unused-function"]


def build(force=False):
    """Compile the oracle with gcc (FP contraction off: the FP32 key path must
    round every operation exactly once)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class OrcCamera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("znear", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


class OrcOpts(C.Structure):
    _fields_ = [("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_min", C.c_float),
                ("bg", C.c_float * 3), ("sh_degree", C.c_int32), ("log_params", C.c_int32),
                ("proj64", C.c_int32), ("mode", C.c_int32), ("flag_margin", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i64 = C.c_int64
            lib.orc_num_threads.restype = C.c_int
            lib.orc_project.argtypes = [i64, P, P, C.POINTER(OrcCamera), C.c_int32, C.c_int32, P, P, P, P, P, P, P]
            lib.orc_radius.argtypes = [i64, P, P, P]
            lib.orc_row_span.argtypes = [i64, P, P, P, P, P, P, C.c_int32, P, P]
            lib.orc_keys.argtypes = [i64, P, P, P, P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint32,
                                     P, P, P]
            lib.orc_keys.restype = i64
            lib.orc_render.argtypes = [i64, P, P, P, C.POINTER(OrcCamera), C.POINTER(OrcOpts), P, P, P, P, P, P]
            lib.orc_render.restype = i64
            lib.orc_backward.argtypes = [i64, P, P, P, C.POINTER(OrcCamera), C.POINTER(OrcOpts), P,
                                         P, P, P, P, P, P, P, P, P, P, P]
            lib.orc_backward.restype = i64
            lib.orc_activate.argtypes = [i64, P, i64, P, P, P]
            lib.orc_sh_basis.argtypes = [C.c_int32, i64, P, P, P]
            lib.orc_l1.argtypes = [i64, P, P, P]
            lib.orc_l1.restype = C.c_double
            lib.orc_adam.argtypes = [i64, P, P, P, P, C.c_double, C.c_double, C.c_double, C.c_double, i64]
            lib.orc_l1_ssim.argtypes = [i64, i64, i64, P, P, C.c_double, P, P, P]
            lib.orc_l1_ssim.restype = C.c_double
            lib.orc_fit2d_render.argtypes = [i64, P, C.c_float, C.c_int32, C.c_int32, P]
            lib.orc_fit2d_backward.argtypes = [i64, P, C.c_float, C.c_int32, C.c_int32, P, P]
            lib.orc_quadtree_init.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P]
            lib.orc_quadtree_init.restype = i64
            lib.orc_fit2d_densify.argtypes = [i64, P, P, P, P, C.c_int32, C.c_float, C.c_float, C.c_float, i64,
                                              P, P, P]
            lib.orc_fit2d_densify.restype = i64
            lib.orc_fit2d_grad_accum.argtypes = [i64, P, P]
            lib.orc_grad_accum3d.argtypes = [i64, P, P, P, P]
            lib.orc_densify3d.argtypes = [i64, C.c_int32, C.c_int32] + [P] * 11 + [C.c_float] * 3 + [i64] + [P] * 9
            lib.orc_densify3d.restype = i64
            lib.orc_merge3d.argtypes = [i64, C.c_int32, C.c_int32] + [P] * 9 + [P, C.c_float, C.c_float] + [P] * 9
            lib.orc_merge3d.restype = i64
            lib.orc_octree_init.argtypes = [i64, P, P, P, C.c_float, C.c_int32, i64, C.c_float, C.c_int32, C.c_int32,
                                            P, P, P]
            lib.orc_octree_init.restype = i64
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().orc_num_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _cam(cam) -> OrcCamera:
    c = OrcCamera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).reshape(9)]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float32).reshape(3)]
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.znear = cam.znear
    c.width, c.height = cam.width, cam.height
    return c


def _opts(scene, mode, proj64, bg, alpha_min, alpha_max, t_min, flag_margin) -> OrcOpts:
    o = OrcOpts()
    o.alpha_min, o.alpha_max, o.t_min = alpha_min, alpha_max, t_min
    o.bg[:] = list(bg)
    o.sh_degree = scene.sh_degree
    o.log_params = int(scene.log_params)
    o.proj64 = int(proj64)
    o.mode = int(mode)
    o.flag_margin = float(flag_margin)
    return o


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# ------------------------------------------------------------ key path ------

def radius(s, o):
    """Footprint radius (Eq. 2's support, per particle) of screen size s and
    opacity o: an FP32 upper bound of s sqrt(2 (ln(255 o) + 2^-9))."""
    s, o = _c32(np.atleast_1d(s)), _c32(np.atleast_1d(o))
    r = np.zeros(s.shape[0], np.float32)
    _load().orc_radius(s.shape[0], _ptr(s), _ptr(o), _ptr(r))
    return r


def project(means_sigma, opacity, cam, tile, footprint=0):
    """Canonical FP32 projection (linear sigma/opacity): u, v, s, r (footprint
    radius), depth, rect (x0, y0, x1, y1 inclusive tile bounds) and tiles
    touched (0 = culled): every tile of rect (footprint 0) or, per row, the
    tiles the disc meets (footprint 1). Eq. 7 with Sigma = sigma^2 I; support
    of Eq. 2."""
    ms, op = _c32(means_sigma), _c32(opacity)
    n = ms.shape[0]
    out = {k: np.zeros(n, np.float32) for k in ("u", "v", "s", "depth", "r")}
    rect = np.zeros((n, 4), np.int32)
    count = np.zeros(n, np.int32)
    _load().orc_project(n, _ptr(ms), _ptr(op), C.byref(_cam(cam)), int(tile), int(footprint), _ptr(out["u"]),
                        _ptr(out["v"]), _ptr(out["s"]), _ptr(out["depth"]), _ptr(out["r"]), _ptr(rect),
                        _ptr(count))
    out["rect"], out["count"] = rect, count
    out["footprint"] = int(footprint)
    return out


def row_span(u, v, r, ty, x0, x1, tile):
    """Tiles [xa, xb] of tile row ty (within [x0, x1]) that the disc of radius r
    around (u, v) touches; empty when xa > xb. Vectorised over the arguments."""
    shape = np.broadcast_shapes(*(np.shape(np.atleast_1d(a)) for a in (u, v, r, ty, x0, x1)))
    u, v, r = (_c32(np.broadcast_to(np.atleast_1d(np.asarray(a, np.float32)), shape).ravel()) for a in (u, v, r))
    ty, x0, x1 = (np.ascontiguousarray(np.broadcast_to(np.atleast_1d(a), shape).ravel(), np.int32)
                  for a in (ty, x0, x1))
    xa = np.zeros(u.shape[0], np.int32)
    xb = np.zeros(u.shape[0], np.int32)
    _load().orc_row_span(u.shape[0], _ptr(u), _ptr(v), _ptr(r), _ptr(ty), _ptr(x0), _ptr(x1), int(tile),
                         _ptr(xa), _ptr(xb))
    return xa, xb


def keys(proj, cam, tile, tile_base=0):
    """Sorted (key, value) pairs and per-tile [start, end) ranges of the
    depth-ordered tile lists: key = tile << 32 | FP32 depth bits (front-to-back
    order of Eq. 4 within each tile, ties by Gaussian index)."""
    tiles_x = (cam.width + tile - 1) // tile
    tiles_y = (cam.height + tile - 1) // tile
    m = int(proj["count"].astype(np.int64).sum())
    k = np.zeros(m, np.uint64)
    v = np.zeros(m, np.uint32)
    r = np.zeros((tiles_x * tiles_y, 2), np.uint32)
    got = _load().orc_keys(proj["count"].shape[0], _ptr(np.ascontiguousarray(proj["rect"])),
                           _ptr(np.ascontiguousarray(proj["count"])),
                           _ptr(np.ascontiguousarray(proj["depth"])), _ptr(np.ascontiguousarray(proj["u"])),
                           _ptr(np.ascontiguousarray(proj["v"])), _ptr(np.ascontiguousarray(proj["r"])),
                           int(tile), int(proj.get("footprint", 0)), tiles_x, tiles_y, int(tile_base), _ptr(k),
                           _ptr(v), _ptr(r))
    assert got == m
    return k, v, r


def activate(log_sigma, logit):
    """sigma = exp(log sigma), opacity = sigmoid(logit), in FP64 then rounded
    once to FP32 (the 4 kernel parameters of Sec. 2.1 kept unconstrained)."""
    ls, lg = _c32(log_sigma), _c32(logit)
    n = ls.shape[0]
    s = np.zeros(n, np.float32)
    o = np.zeros(n, np.float32)
    _load().orc_activate(n, _ptr(ls), 1, _ptr(lg), _ptr(s), _ptr(o))
    return s, o


def sh_basis(deg, dirs):
    """Real orthonormal SH basis (no Condon-Shortley phase) up to ``deg`` at unit
    directions [n, 3] (FP64), with gradients of the polynomial extension."""
    d = np.ascontiguousarray(dirs, np.float64)
    n = d.shape[0]
    K = (deg + 1) ** 2
    Y = np.zeros((n, K))
    dY = np.zeros((n, K, 3))
    _load().orc_sh_basis(int(deg), n, _ptr(d), _ptr(Y), _ptr(dY))
    return Y, dY


# ----------------------------------------------------------- compositing ----

DEFAULTS = dict(bg=(0.0, 0.0, 0.0), alpha_min=1.0 / 255.0, alpha_max=0.99, t_min=1e-4)


def render(scene, cam, *, mode=1, proj64=False, flag_margin=1e-5, bg=(0.0, 0.0, 0.0),
           alpha_min=1.0 / 255.0, alpha_max=0.99, t_min=1e-4):
    """FP64 front-to-back compositing (Eq. 4) of every visible Gaussian at every
    pixel centre, with no tiling. Returns img [3,H,W], T [H,W], nb [H,W] (entries
    blended), last [H,W] (index of the last blended Gaussian, -1 if none),
    flag [H,W] (a cutoff or stop decision within ``flag_margin`` relative of its
    threshold) and hash [H,W] (digest of the decision sequence)."""
    ms, op, col = _c32(scene.means_sigma), _c32(scene.opacity), _c32(scene.color)
    H, W = cam.height, cam.width
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nb = np.zeros((H, W), np.int32)
    last = np.zeros((H, W), np.int32)
    flag = np.zeros((H, W), np.uint8)
    hsh = np.zeros((H, W), np.uint64)
    o = _opts(scene, mode, proj64, bg, alpha_min, alpha_max, t_min, flag_margin)
    nv = _load().orc_render(scene.n, _ptr(ms), _ptr(op), _ptr(col), C.byref(_cam(cam)), C.byref(o),
                            _ptr(img), _ptr(T), _ptr(nb), _ptr(last), _ptr(flag), _ptr(hsh))
    return dict(img=img, T=T, nb=nb, last=last, flag=flag, hash=hsh, n_visible=int(nv))


def backward(scene, cam, dL_dimg, *, mode=1, proj64=False, flag_margin=1e-5, bg=(0.0, 0.0, 0.0),
             alpha_min=1.0 / 255.0, alpha_max=0.99, t_min=1e-4):
    """Forward plus adjoint (Eq. 3 and the position gradient after it, through
    Eq. 4, Eq. 8 and the projection). Gradients are w.r.t. the stored
    parameters: sigma or log sigma, opacity or its logit, RGB or SH."""
    ms, op, col = _c32(scene.means_sigma), _c32(scene.opacity), _c32(scene.color)
    n = scene.n
    H, W = cam.height, cam.width
    G = np.ascontiguousarray(dL_dimg, np.float64).reshape(3, H, W)
    out = dict(d_means=np.zeros((n, 3)), d_sigma=np.zeros(n), d_opac=np.zeros(n),
               d_color=np.zeros(col.shape), g2d=np.zeros((n, 7)),
               img=np.zeros((3, H, W)), T=np.zeros((H, W)), nb=np.zeros((H, W), np.int32),
               last=np.zeros((H, W), np.int32), flag=np.zeros((H, W), np.uint8),
               hash=np.zeros((H, W), np.uint64))
    o = _opts(scene, mode, proj64, bg, alpha_min, alpha_max, t_min, flag_margin)
    nv = _load().orc_backward(n, _ptr(ms), _ptr(op), _ptr(col), C.byref(_cam(cam)), C.byref(o), _ptr(G),
                              _ptr(out["d_means"]), _ptr(out["d_sigma"]), _ptr(out["d_opac"]),
                              _ptr(out["d_color"]), _ptr(out["g2d"]), _ptr(out["img"]), _ptr(out["T"]),
                              _ptr(out["nb"]), _ptr(out["last"]), _ptr(out["flag"]), _ptr(out["hash"]))
    out["n_visible"] = int(nv)
    return out


# ------------------------------------------------------------ loss, Adam ----

def l1(img, target):
    """Mean absolute error over all 3 H W entries and its gradient (the L1 term
    of the loss of Sec. 3, with lambda = 0)."""
    im = np.ascontiguousarray(img, np.float64)
    tg = _c32(target)
    grad = np.zeros(im.shape)
    loss = _load().orc_l1(im.size, _ptr(im), _ptr(tg), _ptr(grad))
    return float(loss), grad


def l1_ssim(img, target, lam=0.2, grad=True, ssim_map=False):
    """The loss of Sec. 3 with its structural term: (1 - lam) mean |img - target|
    + lam (1 - SSIM), SSIM with the 11 x 11 Gaussian window (std 1.5, zero
    outside the image), C1 = 0.01^2, C2 = 0.03^2, per channel of planar
    [channels][height][width] images (a 2-D image is one channel). FP64.
    Returns (loss, ssim, dL/dimg or None), plus the per-entry SSIM if ssim_map."""
    im = np.array(img, np.float64, copy=True)
    tg = np.array(target, np.float64, copy=True)
    if im.shape != tg.shape or im.ndim not in (2, 3):
        raise ValueError("img and target: equal [C][H][W] or [H][W] shapes")
    shp = im.shape if im.ndim == 3 else (1,) + im.shape
    g = np.zeros(im.shape) if grad else None
    ssim = np.zeros(1)
    smap = np.zeros(im.shape) if ssim_map else None
    loss = _load().orc_l1_ssim(shp[0], shp[1], shp[2], _ptr(im), _ptr(tg), float(lam), _ptr(ssim),
                               _ptr(smap) if ssim_map else None, _ptr(g) if grad else None)
    if ssim_map:
        return float(loss), float(ssim[0]), g, smap
    return float(loss), float(ssim[0]), g


def adam(p, grad, m, v, *, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, t=1):
    """One bias-corrected Adam step in FP64, in place on copies; returns (p, m, v)."""
    p = np.array(p, np.float64, copy=True)
    m = np.array(m, np.float64, copy=True)
    v = np.array(v, np.float64, copy=True)
    g = np.ascontiguousarray(grad, np.float64)
    _load().orc_adam(p.size, _ptr(p), _ptr(g), _ptr(m), _ptr(v), lr, b1, b2, eps, int(t))
    return p, m, v


# ------------------------------------------------- 2D additive fitting ----

def fit2d_render(params, D, width, height):
    """The paper's 2D model (Sec. 3): f^(x) = sum over particles with
    |mu_k - x| < D of A_k exp(-|x - mu_k|^2 / (2 sigma_k^2)), the support test in
    canonical FP32, values in FP64. params [K][8] = (mu_x, mu_y, log sigma,
    A_r, A_g, A_b, 0, 0). Returns [3][H][W] float64."""
    p = _c32(params).reshape(-1, 8)
    img = np.zeros((3, height, width))
    _load().orc_fit2d_render(p.shape[0], _ptr(p), float(D), int(width), int(height), _ptr(img))
    return img


def fit2d_backward(params, D, G):
    """Gradient w.r.t. the particles ([K][8], FP64) of a loss whose image
    gradient is G ([3][H][W])."""
    p = _c32(params).reshape(-1, 8)
    g = np.ascontiguousarray(G, np.float64)
    out = np.zeros((p.shape[0], 8))
    _load().orc_fit2d_backward(p.shape[0], _ptr(p), float(D), int(g.shape[2]), int(g.shape[1]), _ptr(g), _ptr(out))
    return out


def quadtree_init(img, k_max, min_cell):
    """QuadTree initialisation (Sec. 3.1) of a square power-of-two RGB image
    ([3][S][S], S <= 512): one particle per leaf at the cell centre, A = the
    cell's mean colour, sigma = half the cell width; the leaf with the largest
    squared error is split while the leaves stay <= k_max and the children are
    >= min_cell wide. Returns [L][8] float32."""
    im = _c32(img)
    if im.ndim != 3 or im.shape[0] != 3 or im.shape[1] != im.shape[2]:
        raise ValueError("img must be [3][S][S]")
    out = np.zeros((max(k_max, 1), 8), np.float32)
    n = _load().orc_quadtree_init(_ptr(im), im.shape[1], int(k_max), int(min_cell), _ptr(out))
    if n < 0:
        raise ValueError("side must be a power of two <= 512, k_max and min_cell >= 1")
    return out[:n].copy()


def fit2d_grad_accum(d_particles, accum):
    """accum_i + |dL/dmu_i| (FP32, one rounding per step) for the 2D particles'
    gradients d_particles [k][8]; returns the new accumulator."""
    g = _c32(d_particles).reshape(-1, 8)
    acc = _c32(accum).reshape(-1).copy()
    if acc.shape[0] != g.shape[0]:
        raise ValueError("accum must hold one value per particle")
    _load().orc_fit2d_grad_accum(g.shape[0], _ptr(g), _ptr(acc))
    return acc


def fit2d_densify(params, m, v, accum, n_iters, tau_a, tau_g, log_sigma_min, capacity):
    """Delete particles with max |A| < tau_a; divide those whose summed
    position-gradient norm exceeds tau_g * n_iters and whose log sigma >=
    log_sigma_min into four sigma/2 children at mu +- sigma/2 (the first
    candidates that fit `capacity`); keep the rest. Returns (params, m, v)."""
    p, mm, vv = _c32(params).reshape(-1, 8), _c32(m).reshape(-1, 8), _c32(v).reshape(-1, 8)
    acc = _c32(accum).reshape(-1)
    out = np.zeros((capacity, 8), np.float32)
    om, ov = np.zeros_like(out), np.zeros_like(out)
    n = _load().orc_fit2d_densify(p.shape[0], _ptr(p), _ptr(mm), _ptr(vv), _ptr(acc), int(n_iters), float(tau_a),
                                  float(tau_g), float(log_sigma_min), int(capacity), _ptr(out), _ptr(om), _ptr(ov))
    return out[:n].copy(), om[:n].copy(), ov[:n].copy()


def grad_accum3d(g2d, count, accum, vis):
    """Densify statistic of the 3D Gaussians after one step: for every Gaussian
    that touched a tile (count > 0), accum += |(du, dv)| (FP32, one rounding per
    step) and vis += 1. Returns (accum, vis)."""
    g = _c32(g2d).reshape(-1, 8)
    cnt = np.ascontiguousarray(count, np.uint32).reshape(-1)
    acc = _c32(accum).reshape(-1).copy()
    vv = np.ascontiguousarray(vis, np.uint32).reshape(-1).copy()
    if not (g.shape[0] == cnt.shape[0] == acc.shape[0] == vv.shape[0]):
        raise ValueError("g2d, count, accum and vis must describe the same Gaussians")
    _load().orc_grad_accum3d(g.shape[0], _ptr(g), _ptr(cnt), _ptr(acc), _ptr(vv))
    return acc, vv


def densify3d(params, m, v, accum, vis, param_mode, op_min, tau_g, scale_min, capacity):
    """Delete (stored opacity < op_min), divide (mean screen-space position
    gradient accum / vis > tau_g and stored scale >= scale_min: eight half-scale
    children, one per octant at mu +- sigma / 2) or keep each 3D Gaussian, within
    `capacity`. params, m, v: (means_sigma [n][4], opacity [n], color [n][C]).
    Returns (params, m, v) of the result, same layout."""
    ms, op, col = (_c32(a) for a in params)
    n = ms.shape[0]
    C = col.reshape(n, -1).shape[1] if n else col.shape[-1]
    col = col.reshape(n, C)
    mm = [_c32(a) for a in m]
    vv = [_c32(a) for a in v]
    acc = _c32(accum).reshape(-1)
    vis_ = np.ascontiguousarray(vis, np.uint32).reshape(-1)
    outs = [np.zeros((capacity, 4), np.float32), np.zeros(capacity, np.float32), np.zeros((capacity, C), np.float32)]
    om = [np.zeros_like(a) for a in outs]
    ov = [np.zeros_like(a) for a in outs]
    k = _load().orc_densify3d(n, C, int(param_mode), _ptr(ms), _ptr(op), _ptr(col), *[_ptr(a) for a in mm],
                              *[_ptr(a) for a in vv], _ptr(acc), _ptr(vis_), float(op_min), float(tau_g),
                              float(scale_min), int(capacity), *[_ptr(a) for a in outs], *[_ptr(a) for a in om],
                              *[_ptr(a) for a in ov])
    cut = lambda arrs: tuple(a[:k].copy() for a in arrs)  # noqa: E731
    return cut(outs), cut(om), cut(ov)


def merge3d(params, m, v, param_mode, lo, h, scale_max):
    """Merging of the 3D Gaussians, read as the inverse of the octant division
    (Sec. 3.2, 2.5, 3.1): the eligible Gaussians (finite mean, stored scale <=
    scale_max, opacity >= 2^-60, cell of side h from lo within 1024 per axis) that
    share a cell, two or more of them, become one Gaussian at the place of the
    first (opacity-weighted mean and colour, moment-matched isotropic scale,
    opacity min(0.99, 1 - prod (1 - o_k)), zero moments); the rest are kept.
    params, m, v: (means_sigma [n][4], opacity [n], color [n][C]); returns
    (params, m, v) of the result in index order."""
    ms, op, col = (_c32(a) for a in params)
    n = ms.shape[0]
    C = col.reshape(n, -1).shape[1] if n else col.shape[-1]
    col = col.reshape(n, C)
    mm = [_c32(a) for a in m]
    vv = [_c32(a) for a in v]
    lo3 = _c32(np.asarray(lo, np.float32).reshape(3))
    outs = [np.zeros((max(n, 1), 4), np.float32), np.zeros(max(n, 1), np.float32), np.zeros((max(n, 1), C), np.float32)]
    om = [np.zeros_like(a) for a in outs]
    ov = [np.zeros_like(a) for a in outs]
    k = _load().orc_merge3d(n, C, int(param_mode), _ptr(ms), _ptr(op), _ptr(col), *[_ptr(a) for a in mm],
                            *[_ptr(a) for a in vv], _ptr(lo3), float(h), float(scale_max), *[_ptr(a) for a in outs],
                            *[_ptr(a) for a in om], *[_ptr(a) for a in ov])
    cut = lambda arrs: tuple(a[:k].copy() for a in arrs)  # noqa: E731
    return cut(outs), cut(om), cut(ov)


def octree_init(points, colors, lo, side, levels, k_max, opacity=0.5, sh_degree=-1, param_mode=0):
    """Octree initialisation of 3D Gaussians from a coloured point set: greedy
    splits of the leaf with the largest squared colour error (12-bit exact
    statistics) while the non-empty leaves stay <= k_max; one Gaussian per
    non-empty leaf (cell centre, sigma = half the cell side, mean colour).
    Returns (means_sigma [K][4], opacity [K], color [K][C])."""
    p = _c32(points).reshape(-1, 3)
    c = _c32(colors).reshape(-1, 3)
    lo3 = _c32(np.asarray(lo, np.float32).reshape(3))
    C = 3 if sh_degree < 0 else 3 * (sh_degree + 1) ** 2
    cap = max(int(k_max), 1)
    ms = np.zeros((cap, 4), np.float32)
    op = np.zeros(cap, np.float32)
    col = np.zeros((cap, C), np.float32)
    k = _load().orc_octree_init(p.shape[0], _ptr(p), _ptr(c), _ptr(lo3), float(side), int(levels), int(k_max),
                                float(opacity), int(sh_degree), int(param_mode), _ptr(ms), _ptr(op), _ptr(col))
    if k < 0:
        raise ValueError("need 0 <= levels <= 7, k_max >= 1, side > 0, sh_degree in -1..3")
    return ms[:k].copy(), op[:k].copy(), col[:k].copy()
