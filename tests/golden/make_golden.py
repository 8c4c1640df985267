"""Writes tests/golden/oracle_tiny.json from the CPU oracle alone.

The paper (arXiv 2403.14244) prints no worked numerical example for the
rasteriser, so the stored values here are the oracle's own output on a tiny
seeded scene: a regression guard. Any change to the oracle's arithmetic that
moves them must be justified by the passage of the paper (or the reading of it)
that requires it, and this script re-run.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from tests._tiny import random_small  # noqa: E402

PIXELS = [(3, 2), (10, 7), (12, 9), (15, 5), (20, 11), (8, 12)]


def make():
    sc, cam = random_small(40, 1234, w=24, h=16, sh_degree=3, spread=0.5)
    out = oracle.render(sc, cam, mode=0)
    W = np.ones((3, cam.height, cam.width))
    g = oracle.backward(sc, cam, W, mode=0)
    p = oracle.project(sc.means_sigma, sc.opacity, cam, 8)
    k, v, r = oracle.keys(p, cam, 8)
    return {
        "source": "oracle/igs_oracle.c on tests/_tiny.random_small(40, 1234, w=24, h=16, sh_degree=3, spread=0.5)",
        "equations": "Eq. 4 compositing, Eq. 8 kernel, Eq. 7 with Sigma = sigma^2 I; gradients by Eq. 3",
        "pixels": [{"x": x, "y": y, "rgb": [float(out["img"][c, y, x]) for c in range(3)],
                    "T": float(out["T"][y, x]), "nb": int(out["nb"][y, x])} for x, y in PIXELS],
        "keys_tile8_first16": [int(x) for x in k[:16]],
        "vals_tile8_first16": [int(x) for x in v[:16]],
        "M_tile8": int(len(k)),
        "sum_d_means": [float(x) for x in g["d_means"].sum(axis=0)],
        "sum_d_color": float(g["d_color"].sum()),
    }


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny.json")
    with open(path, "w") as f:
        json.dump(make(), f, indent=1)
    print("wrote", path)
