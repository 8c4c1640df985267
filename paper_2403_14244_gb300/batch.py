"""Batched multi-view rendering, captured in a CUDA graph, with an autotuner.

``BatchRenderer`` renders many views of one scene (mixed image sizes) through
igs_render_batch: views are packed into groups whose (view, Gaussian, tile)
entries fit one batch workspace (the entry budget), each view gets a frame
sized from a calibrating render of it, each group is one chain of launches
(one projection launch, the views' binnings on concurrent streams, one blend
launch), the groups' chains run on streams of their own (so one group's blend
overlaps another's binnings), and all of it is captured once in a CUDA graph
and replayed for each new set of poses.

``autotune`` times every supported (tile size, blend staging depth) pair on the
caller's workload and caches the fastest, keyed by the workload's shape.
"""
from __future__ import annotations

import json
import math
import os
import time

import torch

from . import igs
from .render import Renderer

DEFAULT_ENTRY_BUDGET = 300_000_000
BLEND_BATCHES = {8: (32, 64), 16: (64, 128, 256), 32: (64, 256, 512, 1024)}  # 64 at 16 and 32: sub-tile blend


def views_entries(scene: igs.Scene, cams, tile, sh_degree, param_mode=0, device="cuda", footprint=0):
    """Entries each view needs (one binning pass per view, synchronising)."""
    r = Renderer(tile=tile, sh_degree=sh_degree, param_mode=param_mode, device=device, footprint=footprint)
    out = []
    for c in cams:
        _, f = r.run_forward(scene, c, check=True)
        st, info = igs.frame_status(f)
        out.append(int(info[0]))
    return out


def pack_groups(entries, budget):
    """Consecutive groups of views whose entries sum to at most `budget`."""
    groups, cur, tot = [], [], 0
    for v, m in enumerate(entries):
        if cur and tot + m > budget:
            groups.append(cur)
            cur, tot = [], 0
        cur.append(v)
        tot += m
    if cur:
        groups.append(cur)
    return groups


class BatchRenderer:
    def __init__(self, scene: igs.Scene, cams, tile=16, blend_batch=0, sh_degree=-1, param_mode=0,
                 bg=(0.0, 0.0, 0.0), entry_budget=DEFAULT_ENTRY_BUDGET, margin=1.10, device="cuda", footprint=0):
        self.scene = scene
        self.cams = [c if isinstance(c, igs.IgsCamera) else igs.camera(c) for c in cams]
        self.opts = igs.opts(tile=tile, sh_degree=sh_degree, param_mode=param_mode, bg=bg, footprint=footprint)
        self.tile, self.blend_batch = tile, blend_batch
        self.device = device
        ent = views_entries(scene, self.cams, tile, sh_degree, param_mode, device, footprint)
        self.entries = ent
        cap_budget = min(entry_budget, int(((1 << 30) - 1) / margin) - 65536)
        self.groups = pack_groups([int(m * margin) + 65536 for m in ent], cap_budget)
        self.batches = []
        for g in self.groups:
            caps = [int(ent[v] * margin) + 65536 for v in g]
            b = igs.Batch(scene.n, [self.cams[v] for v in g], self.opts, caps, blend_batch, device)
            b.set_views()
            self.batches.append(b)
        self.graph = None
        self.stream = torch.cuda.Stream(device=device)

    def render(self, stream=None):
        """Render every group (no host synchronisation); groups run concurrently."""
        main = stream if stream is not None else torch.cuda.current_stream(self.device)
        if len(self.batches) == 1:
            self.batches[0].render(self.scene, main)
            return
        if not hasattr(self, "_gstreams"):
            self._gstreams = [torch.cuda.Stream(device=self.device) for _ in self.batches]
        for s in self._gstreams:
            s.wait_stream(main)
        for b, s in zip(self.batches, self._gstreams):
            b.render(self.scene, s)
        for s in self._gstreams:
            main.wait_stream(s)

    def set_poses(self, cams, stream=None):
        """New poses (same image sizes, same order); effective for the next render or replay."""
        self.cams = [c if isinstance(c, igs.IgsCamera) else igs.camera(c) for c in cams]
        for g, b in zip(self.groups, self.batches):
            b.set_views([self.cams[v] for v in g], stream)

    def check(self):
        """Status of every group after a render; raises on a device error."""
        for b in self.batches:
            st, info = b.status()
            if st != igs.OK:
                raise igs.IgsError(st, f"batch render failed (entries needed {info[3]}, capacity {b.capacity})")

    def capture(self):
        """Capture one render of all groups in a CUDA graph (after one eager render)."""
        s = self.stream
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.render(s)
        torch.cuda.synchronize()
        self.check()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.render(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def image(self, v):
        for g, b in zip(self.groups, self.batches):
            if v in g:
                return b.image(g.index(v))
        raise IndexError(v)


def workload_key(scene: igs.Scene, cams, sh_degree):
    sizes = sorted((int(c.width), int(c.height)) for c in cams)
    nb = 2 ** int(round(math.log2(max(scene.n, 1))))
    return f"n~{nb}|sh{sh_degree}|views{len(cams)}|" + ",".join(f"{w}x{h}" for w, h in sizes)


def default_cache_path():
    return os.environ.get("IGS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "igs", "autotune.json"))


def autotune(scene: igs.Scene, cams, sh_degree=-1, candidates=None, reps=5, cache_path=None, use_cache=True,
             device="cuda"):
    """Time every (tile, blend staging depth) candidate on this workload (graph
    replays, CUDA events) and return (best, timings). The result is cached in a
    JSON file keyed by the workload's shape."""
    cache_path = cache_path or default_cache_path()
    key = workload_key(scene, cams, sh_degree)
    cache = {}
    if os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        e = cache[key]
        return (e["tile"], e["blend_batch"]), e["timings_ms"]
    if candidates is None:
        candidates = [(t, b) for t, bs in BLEND_BATCHES.items() for b in bs]
    timings = {}
    for tile, bb in candidates:
        br = BatchRenderer(scene, cams, tile=tile, blend_batch=bb, sh_degree=sh_degree, device=device)
        br.capture()
        br.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            br.replay()
        b.record()
        torch.cuda.synchronize()
        timings[f"{tile}/{bb}"] = a.elapsed_time(b) / reps
        del br
        torch.cuda.empty_cache()
    best = min(timings, key=timings.get)
    tile, bb = (int(x) for x in best.split("/"))
    cache[key] = {"tile": tile, "blend_batch": bb, "timings_ms": timings, "when": time.time()}
    os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
    tmp = cache_path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, cache_path)
    return (tile, bb), timings
