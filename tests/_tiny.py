"""Tiny hand-built scenes for the oracle pins (inputs only, no method arithmetic)."""
import numpy as np

from paper_2403_14244_gb300 import scenes


def scene_from(means, sigma, opac, color, sh_degree=-1, log_params=False):
    n = len(sigma)
    ms = np.zeros((n, 4), np.float32)
    ms[:, :3] = np.asarray(means, np.float64).reshape(n, 3)
    ms[:, 3] = np.asarray(sigma, np.float64)
    C = 3 if sh_degree < 0 else 3 * (sh_degree + 1) ** 2
    return scenes.Scene(means_sigma=ms, opacity=np.asarray(opac, np.float32).reshape(n),
                        color=np.ascontiguousarray(np.asarray(color, np.float32).reshape(n, C)),
                        sh_degree=sh_degree, log_params=log_params)


def small_camera(w=16, h=16, f=64.0, cx=None, cy=None, center=(0.0, 0.0, -4.0)):
    return scenes.pinhole(center, w, h, f, cx, cy)


def random_small(n, seed, w=24, h=20, sh_degree=-1, log_params=False, spread=0.5, smin=0.03, smax=0.15):
    """n Gaussians in a small box in front of a w x h camera, footprints of a few pixels."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-spread, spread, size=(n, 3))
    sigma = np.exp(rng.uniform(np.log(smin), np.log(smax), size=n))
    opac = rng.uniform(0.1, 0.95, size=n)
    if sh_degree < 0:
        color = rng.uniform(0, 1, size=(n, 3))
    else:
        K = (sh_degree + 1) ** 2
        color = rng.normal(0, 0.3, size=(n, K, 3))
        color[:, 0, :] = rng.uniform(-1, 1, size=(n, 3))
    if log_params:
        sigma_col = np.log(sigma)
        opac = np.log(opac / (1 - opac))
    else:
        sigma_col = sigma
    sc = scene_from(means, sigma_col, opac, color.reshape(n, -1), sh_degree, log_params)
    cam = scenes.pinhole((0.3, -0.2, -3.0), w, h, 40.0)
    return sc, cam
