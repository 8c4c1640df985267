"""Seeded synthetic scenes, cameras and targets.

This module only draws inputs: it holds none of the splatting arithmetic
(no projection, no compositing, no gradients). Both the CUDA path and the CPU
oracle consume what it produces, so the two sides see the same bytes.

The paper (arXiv 2403.14244) ships no dataset, images or trained weights, and
its only experiment is a 2D image fit whose image is missing. All inputs here
are synthetic, with the sizes and distributions of the five workloads the hot
path is measured on:

* ``uniform``   means U[-1,1]^3, sigma log-uniform [0.005, 0.05], opacity
                U[0.05, 0.95], RGB U[0,1]                (4096 / 2M / 3M ...)
* ``clustered`` 70 % of the means from 64 Gaussian clusters (centres
                U[-1,1]^3, std U[0.05,0.3]) and 30 % on the unit sphere;
                sigma = exp(N(ln 0.01, 0.7)); opacity = sigmoid(N(0, 1.5^2));
                degree-3 SH with DC U[-1,1] and the rest N(0, 0.1^2)

All arrays are float32 and C-contiguous. Layout (structure of arrays):

* ``means_sigma``  float32 [N, 4]  (x, y, z, sigma or log sigma)
* ``opacity``      float32 [N]     (opacity or its logit)
* ``color``        float32 [N, C]  C = 3 (RGB) or 48 (SH degree 3 stored
                                   coefficient-major: color[i, 3*k + ch])

Cameras follow the pinhole model x_c = R x_w + t with image x to the right,
y down and z forward; world +y is "down", so the camera at (0, 0, -4) looking
at the origin has R = I and t = (0, 0, 4).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

Y00 = 0.28209479177387814  # 1 / (2 sqrt(pi)): the constant l = 0 SH basis function


@dataclasses.dataclass
class Camera:
    R: np.ndarray          # float32 [3, 3], world -> camera rotation (row-major)
    t: np.ndarray          # float32 [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float = 0.01

    def center(self) -> np.ndarray:
        """Camera centre in world coordinates, -R^T t (float64)."""
        return -(self.R.astype(np.float64).T @ self.t.astype(np.float64))


@dataclasses.dataclass
class Scene:
    means_sigma: np.ndarray   # float32 [N, 4]
    opacity: np.ndarray       # float32 [N]
    color: np.ndarray         # float32 [N, C]
    sh_degree: int            # -1 for plain RGB, else 0..3
    log_params: bool = False  # True: column 3 holds log sigma, opacity holds the logit

    @property
    def n(self) -> int:
        return int(self.means_sigma.shape[0])


def look_at(center, target=(0.0, 0.0, 0.0), down=(0.0, 1.0, 0.0)):
    """World->camera (R, t) for a camera at ``center`` looking at ``target``.

    Rows of R are the camera axes in world coordinates: z forward, y the
    component of ``down`` orthogonal to z, x = y cross z (right-handed).
    """
    c = np.asarray(center, np.float64)
    z = np.asarray(target, np.float64) - c
    z /= np.linalg.norm(z)
    d = np.asarray(down, np.float64)
    y = d - (d @ z) * z
    if np.linalg.norm(y) < 1e-6:              # looking straight along "down"
        d = np.array([0.0, 0.0, 1.0])
        y = d - (d @ z) * z
    y /= np.linalg.norm(y)
    x = np.cross(y, z)
    R = np.stack([x, y, z]).astype(np.float64)
    t = -R @ c
    return R.astype(np.float32), t.astype(np.float32)


def pinhole(center, width, height, f, cx=None, cy=None, znear=0.01):
    R, t = look_at(center)
    return Camera(R=R, t=t, fx=float(f), fy=float(f),
                  cx=float(width / 2 if cx is None else cx),
                  cy=float(height / 2 if cy is None else cy),
                  width=int(width), height=int(height), znear=float(znear))


# ---------------------------------------------------------------- scenes ----

def uniform_scene(n, seed, sh_degree=-1, log_params=False):
    """Means U[-1,1]^3, sigma log-uniform [0.005,0.05], opacity U[0.05,0.95],
    RGB U[0,1]. With ``sh_degree`` >= 0 the colour becomes SH with
    DC = (rgb - 0.5) / Y00 and every higher coefficient 0."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(n, 3))
    sigma = np.exp(rng.uniform(math.log(0.005), math.log(0.05), size=n))
    opac = rng.uniform(0.05, 0.95, size=n)
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    return _pack(means, sigma, opac, rgb, sh_degree, log_params)


def clustered_scene(n, seed, sh_degree=3, log_params=False):
    """64-cluster mixture (70 %) plus unit-sphere shell (30 %); log-normal
    sigma; sigmoid-normal opacity; degree-3 SH (DC U[-1,1], rest N(0,0.1^2))."""
    rng = np.random.default_rng(seed)
    n_cl = int(round(0.7 * n))
    centers = rng.uniform(-1.0, 1.0, size=(64, 3))
    stds = rng.uniform(0.05, 0.3, size=64)
    which = rng.integers(0, 64, size=n_cl)
    pts_cl = centers[which] + rng.normal(size=(n_cl, 3)) * stds[which, None]
    sph = rng.normal(size=(n - n_cl, 3))
    sph /= np.linalg.norm(sph, axis=1, keepdims=True)
    means = np.concatenate([pts_cl, sph], axis=0)
    means = means[rng.permutation(n)]
    sigma = np.exp(rng.normal(math.log(0.01), 0.7, size=n))
    opac = 1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.5, size=n)))
    if sh_degree < 0:
        rgb = rng.uniform(0.0, 1.0, size=(n, 3))
        return _pack(means, sigma, opac, rgb, -1, log_params)
    k = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.1, size=(n, k, 3))
    sh[:, 0, :] = rng.uniform(-1.0, 1.0, size=(n, 3))
    return _pack_sh(means, sigma, opac, sh, sh_degree, log_params)


def _pack(means, sigma, opac, rgb, sh_degree, log_params):
    if sh_degree < 0:
        color = rgb
    else:
        k = (sh_degree + 1) ** 2
        sh = np.zeros((rgb.shape[0], k, 3))
        sh[:, 0, :] = (rgb - 0.5) / Y00
        color = sh
    return _pack_sh(means, sigma, opac, color, sh_degree, log_params)


def _pack_sh(means, sigma, opac, color, sh_degree, log_params):
    n = means.shape[0]
    ms = np.empty((n, 4), np.float32)
    ms[:, :3] = means
    if log_params:
        ms[:, 3] = np.log(sigma)
        op = np.log(opac / (1.0 - opac)).astype(np.float32)
    else:
        ms[:, 3] = sigma
        op = opac.astype(np.float32)
    col = np.ascontiguousarray(color.reshape(n, -1), dtype=np.float32)
    return Scene(means_sigma=np.ascontiguousarray(ms), opacity=np.ascontiguousarray(op),
                 color=col, sh_degree=sh_degree, log_params=log_params)


def target_image(width, height, seed):
    """Seeded U[0,1] target image, float32 [3, H, W]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(3, height, width)).astype(np.float32)


# ------------------------------------------------------------- workloads ----

def ring_cameras(k, radius, width, height, f, cx=None, cy=None):
    cams = []
    for i in range(k):
        a = 2.0 * math.pi * i / k
        cams.append(pinhole((radius * math.cos(a), 0.0, radius * math.sin(a)),
                            width, height, f, cx, cy))
    return cams


RESOLUTIONS_BATCH = ((640, 360), (1280, 720), (1920, 1080), (2560, 1440))
RESOLUTIONS_SERVE = ((854, 480), (1280, 720), (1920, 1080), (2560, 1440), (3840, 2160))


def sphere_cameras(k, seed, resolutions=RESOLUTIONS_BATCH, rmin=3.0, rmax=5.0):
    """Cameras at rho * u (u uniform on S^2, rho ~ U[rmin, rmax]) looking at
    the origin; resolution uniform over ``resolutions``; fx = fy = 0.866 W."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(k):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        rho = rng.uniform(rmin, rmax)
        w, h = resolutions[int(rng.integers(0, len(resolutions)))]
        cams.append(pinhole(rho * u, w, h, 0.866 * w))
    return cams


def workload_forward_4k(seed=1):
    """4,096 Gaussians, 256x256, one camera at (0,0,-4), fx = fy = 256."""
    scene = uniform_scene(4096, seed)
    cam = pinhole((0.0, 0.0, -4.0), 256, 256, 256.0)
    return scene, cam


def workload_fwd_bwd_1m(seed=2, n=1_000_000):
    """1M clustered Gaussians with SH degree 3, 1920x1080, fx = fy = 1100,
    seeded U[0,1] target (seed 102)."""
    scene = clustered_scene(n, seed)
    cam = pinhole((0.0, 0.0, -4.0), 1920, 1080, 1100.0)
    target = target_image(1920, 1080, 100 + seed)
    return scene, cam, target


def workload_train_3m(seed=3, n=3_000_000, views=16):
    """3M uniform Gaussians, SH degree 3 (DC from RGB), log sigma and logit
    opacity; 16 ring cameras at radius 4; 1297x840, fx = fy = 1100; per-view
    U[0,1] targets (seed 300 + k)."""
    scene = uniform_scene(n, seed, sh_degree=3, log_params=True)
    cams = ring_cameras(views, 4.0, 1297, 840, 1100.0, cx=648.5, cy=420.0)
    return scene, cams


def train_target(k, width=1297, height=840):
    return target_image(width, height, 300 + k)


# ------------------------------------------------ 2D image-fitting inputs ----

def fit2d_image(side=512, seed=6):
    """Seeded synthetic RGB image, float32 [3, side, side] in [0, 1], standing
    in for the paper's 2D test image (not available): a smooth colour gradient,
    20 filled discs and 12 axis-aligned rectangles of random colours (sharp
    edges at many scales), a sinusoidal texture patch and mild pixel noise."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid((np.arange(side) + 0.5) / side, (np.arange(side) + 0.5) / side, indexing="ij")
    c0, c1 = rng.uniform(0.1, 0.9, size=(2, 3))
    img = np.empty((3, side, side))
    for c in range(3):
        img[c] = c0[c] * (1 - xx) * (1 - yy) + c1[c] * xx * yy + 0.3 * (xx * (1 - yy))
    for _ in range(20):
        cx, cy = rng.uniform(0, 1, size=2)
        r = rng.uniform(0.02, 0.15)
        col = rng.uniform(0, 1, size=3)
        m = (xx - cx) ** 2 + (yy - cy) ** 2 < r * r
        img[:, m] = col[:, None]
    for _ in range(12):
        x0, y0 = rng.uniform(0, 0.9, size=2)
        w, h = rng.uniform(0.03, 0.25, size=2)
        col = rng.uniform(0, 1, size=3)
        m = (xx >= x0) & (xx < x0 + w) & (yy >= y0) & (yy < y0 + h)
        img[:, m] = col[:, None]
    px, py, pw = rng.uniform(0.1, 0.6), rng.uniform(0.1, 0.6), 0.3
    m = (xx >= px) & (xx < px + pw) & (yy >= py) & (yy < py + pw)
    tex = 0.5 + 0.4 * np.sin(2 * np.pi * 24 * xx) * np.sin(2 * np.pi * 17 * yy)
    img[:, m] = tex[m][None, :] * rng.uniform(0.3, 1.0, size=(3, 1))
    img += rng.normal(0.0, 0.01, size=img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def fit2d_particles(k, side, seed, sigma=(1.0, 12.0)):
    """Seeded random 2D particles [k][8] = (mu_x, mu_y, log sigma, A_r, A_g,
    A_b, 0, 0): centres uniform over the image, sigma log-uniform, A ~ U[0, 1]."""
    rng = np.random.default_rng(seed)
    p = np.zeros((k, 8), np.float32)
    p[:, 0:2] = rng.uniform(0.0, side, size=(k, 2))
    p[:, 2] = rng.uniform(np.log(sigma[0]), np.log(sigma[1]), size=k)
    p[:, 3:6] = rng.uniform(0.0, 1.0, size=(k, 3))
    return p


def point_cloud(n, seed=8, clusters=64, spread=0.05):
    """Seeded coloured point set for the Octree initialisation: half the points
    from `clusters` Gaussian clusters (centres U[-0.8, 0.8]^3, std `spread`),
    half uniform in [-1, 1]^3; colours with structure at several scales (two
    smooth waves and a step in z) plus N(0, 0.03^2) noise, clipped to [0, 1].
    Returns (points float32 [n, 3], colours float32 [n, 3])."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-0.8, 0.8, (clusters, 3))
    p = np.concatenate([centres[rng.integers(0, clusters, n // 2)] + rng.normal(0, spread, (n // 2, 3)),
                        rng.uniform(-1, 1, (n - n // 2, 3))]).astype(np.float32)
    c = np.clip(np.stack([0.5 + 0.4 * np.sin(4 * p[:, 0]), 0.5 + 0.4 * np.cos(6 * p[:, 1] * p[:, 2]),
                          (p[:, 2] > 0.1) * 0.7 + 0.15], 1) + rng.normal(0, 0.03, (n, 3)), 0, 1).astype(np.float32)
    return p, c
