"""One-view rendering and training on top of the C ABI.

``Renderer`` chains igs_project -> igs_bin_sort -> igs_render_fwd for a view,
keeps one frame workspace per image size, and sizes the (Gaussian, tile) entry
capacity from the last frame it saw (a frame that overflows reports the entries
it needed and is redone with room to spare). ``IGSRender`` is the
torch.autograd.Function over the same path: each of its forwards leases a frame
of its own from the renderer's pool, so several renders of one image size can
wait for one backward; ``TrainStep`` is one forward + L1 + backward + Adam step
with no host synchronisation except the optional loss read.
"""
from __future__ import annotations

import math
import weakref

import torch

from . import igs

DEFAULT_MIN_CAPACITY = 1 << 16


class Renderer:
    def __init__(self, tile=16, sh_degree=-1, param_mode=0, bg=(0.0, 0.0, 0.0), alpha_min=1.0 / 255.0,
                 alpha_max=0.99, t_min=1e-4, device="cuda", footprint=0):
        self.opts = igs.opts(tile=tile, sh_degree=sh_degree, param_mode=param_mode, alpha_min=alpha_min,
                             alpha_max=alpha_max, t_min=t_min, bg=bg, footprint=footprint)
        self.device = device
        self._frames = {}
        self._cap_hint = {}
        self._free = {}  # frames returned to the lease pool, per (n, width, height)

    def frame(self, n, cam, capacity):
        """The renderer's shared frame of this size: every call of that size
        reuses it (run_forward, TrainStep)."""
        key = (n, cam.width, cam.height)
        f = self._frames.get(key)
        if f is None or f.capacity < capacity:
            f = igs.Frame(n, capacity, cam, self.opts, self.device)
            self._frames[key] = f
        f.cam = cam
        return f

    def lease(self, n, cam, capacity):
        """A frame that no other caller holds until release(): a free pooled frame
        of this size with enough capacity, else a new one. Each lease bumps the
        frame's generation, so a holder can tell whether it was leased again."""
        free = self._free.get((n, cam.width, cam.height), [])
        f = None
        while free and f is None:
            cand = free.pop()
            if cand.capacity >= capacity:
                f = cand  # (too small ones are dropped)
        if f is None:
            f = igs.Frame(n, capacity, cam, self.opts, self.device)
            f.generation = 0
        f.cam = cam
        f.generation += 1
        f.leased = True
        return f

    def release(self, frame, generation=None):
        """Return a leased frame to the pool (no-op if it is not leased, or if
        `generation` is given and the frame has been leased again since)."""
        if not getattr(frame, "leased", False):
            return
        if generation is not None and frame.generation != generation:
            return
        frame.leased = False
        self._free.setdefault((frame.n, frame.width, frame.height), []).append(frame)

    def capacity_for(self, n, cam):
        key = (n, cam.width, cam.height)
        hint = self._cap_hint.get(key)
        if hint is None:
            # first frame of this size: a generous guess, corrected after the fact
            hint = max(DEFAULT_MIN_CAPACITY, 16 * n)
        return int(min(hint, (1 << 30) - 1))

    def note_needed(self, n, cam, needed):
        """Remember the entries a view of this size needed; the capacity only grows."""
        key = (n, cam.width, cam.height)
        want = int(min(math.ceil(needed * 1.15) + 4096, (1 << 30) - 1))
        self._cap_hint[key] = max(want, self._cap_hint.get(key, 0))

    def run_forward(self, scene: igs.Scene, cam, img=None, check=True, stream=None, lease=False):
        """project + bin_sort + render_fwd. Returns (img [3,H,W], frame). With
        check=True the stream is synchronised to read the frame status, and an
        overflowing frame is redone with the capacity it reported. With
        lease=True the frame is leased (release() it when done); otherwise it
        is the renderer's shared frame of this size, which the next call of the
        same size overwrites."""
        c = cam if isinstance(cam, igs.IgsCamera) else igs.camera(cam)
        if img is None:
            img = torch.empty((3, c.height, c.width), dtype=torch.float32, device=self.device)
        for _ in range(3):
            cap = self.capacity_for(scene.n, c)
            f = self.lease(scene.n, c, cap) if lease else self.frame(scene.n, c, cap)
            igs.project(scene, c, self.opts, f, stream)
            f.proj_gen = getattr(f, "proj_gen", 0) + 1  # the frame's projection arrays changed
            igs.bin_sort(f, self.opts, stream)
            igs.render_fwd(f, self.opts, img, stream)
            if not check:
                return img, f
            st, info = igs.frame_status(f, stream)
            if st == igs.OK:
                self.note_needed(scene.n, c, max(info[0], 1))
                return img, f
            if lease:
                self.release(f)
            if st != igs.ERR_CAPACITY:
                raise igs.IgsError(st, "device error during render")
            self.note_needed(scene.n, c, info[3])
        raise igs.IgsError(igs.ERR_CAPACITY, "entry capacity kept overflowing")

    def run_backward(self, scene: igs.Scene, cam, frame, dL_dimg, grads=None, stream=None):
        """Gradients w.r.t. means_sigma [N,4], opacity [N], color [N,C] (overwritten)."""
        c = cam if isinstance(cam, igs.IgsCamera) else igs.camera(cam)
        n = scene.n
        if grads is None:
            grads = (torch.empty_like(scene.means_sigma), torch.empty_like(scene.opacity),
                     torch.empty_like(scene.color))
        g2d = torch.empty((n, 8), dtype=torch.float32, device=self.device)
        igs.render_bwd(scene, c, self.opts, frame, dL_dimg.contiguous(), g2d, *grads, stream)
        return grads


class _FrameLease:
    """A forward's hold on its leased frame; the frame goes back to the pool when
    the backward has used it or when the autograd graph that owns this object
    is freed, whichever comes first."""

    __slots__ = ("frame", "generation", "__weakref__")

    def __init__(self, renderer, frame):
        self.frame, self.generation = frame, frame.generation
        weakref.finalize(self, renderer.release, frame, frame.generation)


class IGSRender(torch.autograd.Function):
    """img = render(means_sigma, opacity, color; camera) with the CUDA adjoint.

    The forward saves its frame (depth order, tile lists, per-pixel T_final and
    contributor counts) for the backward, which walks those lists back to front
    without re-running the forward. Every forward leases its own frame, so
    several views of one size can be rendered into one loss before backward()."""

    @staticmethod
    def forward(ctx, means_sigma, opacity, color, renderer: Renderer, cam):
        scene = igs.Scene(means_sigma.contiguous(), opacity.contiguous(), color.contiguous())
        img, frame = renderer.run_forward(scene, cam, check=True, lease=True)
        ctx.renderer, ctx.cam = renderer, cam
        ctx.lease = _FrameLease(renderer, frame)
        ctx.save_for_backward(means_sigma, opacity, color)
        return img

    @staticmethod
    def backward(ctx, dimg):
        means_sigma, opacity, color = ctx.saved_tensors  # (checks that no input changed in place)
        lease = ctx.lease
        if lease.frame.generation != lease.generation:
            raise RuntimeError("IGSRender: this render's frame was reused by a later forward; a second "
                               "backward through the same graph needs its forward run again")
        scene = igs.Scene(means_sigma.contiguous(), opacity.contiguous(), color.contiguous())
        d_ms, d_op, d_col = ctx.renderer.run_backward(scene, ctx.cam, lease.frame, dimg.contiguous())
        ctx.renderer.release(lease.frame, lease.generation)
        return d_ms, d_op, d_col, None, None


def render(means_sigma, opacity, color, renderer: Renderer, cam):
    return IGSRender.apply(means_sigma, opacity, color, renderer, cam)


class TrainStep:
    """Training state for one scene: a flat FP32 parameter buffer holding
    means_sigma [N,4] (log sigma), opacity [N] (logit) and color [N,C] (SH) as
    views, each segment starting on a 256-byte boundary, and the Adam moments m, v
    in flat buffers of the same layout.

    step(cam, target) runs forward, loss, backward and Adam on the GPU. The loss
    is L1 (ssim_lambda = 0) or the paper's (1 - lambda) L1 + lambda (1 - SSIM)
    (ssim_lambda = lambda, 0.2 in the paper). By default the projection backward
    and Adam run as one fused kernel and the gradient is never written;
    fused=False writes the gradient to `grad` and applies igs_adam over the flat
    buffer (same update)."""

    def __init__(self, means_sigma, opacity, color, sh_degree, tile=16, lr=1e-3, device="cuda", fused=True,
                 footprint=0, ssim_lambda=0.0):
        n = means_sigma.shape[0]
        C = color.shape[1]
        self.n, self.C = n, C
        a = lambda x: (x + 63) // 64 * 64  # noqa: E731  (floats per 256 bytes)
        self.o_op = a(4 * n)
        self.o_col = a(self.o_op + n)
        size = a(self.o_col + C * n)
        self.flat = torch.zeros(size, dtype=torch.float32, device=device)
        self.grad = torch.zeros_like(self.flat)
        self.m = torch.zeros_like(self.flat)
        self.v = torch.zeros_like(self.flat)
        self.ms, self.op, self.col = self._views(self.flat)
        self.g_ms, self.g_op, self.g_col = self._views(self.grad)
        self.m_views = self._views(self.m)
        self.v_views = self._views(self.v)
        self.ms.copy_(means_sigma)
        self.op.copy_(opacity)
        self.col.copy_(color)
        self.scene = igs.Scene(self.ms, self.op, self.col)
        self.renderer = Renderer(tile=tile, sh_degree=sh_degree, param_mode=1, device=device, footprint=footprint)
        self.g2d = torch.empty((n, 8), dtype=torch.float32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        if not 0.0 <= ssim_lambda <= 1.0:
            raise ValueError("ssim_lambda must be in [0, 1]")
        self.ssim_lambda = float(ssim_lambda)
        self._work = {}
        self.lr = lr
        self.fused = fused
        self.t = 0
        self._img = {}
        self._dimg = {}
        self.sh_degree = sh_degree
        self.device = device
        self.tile, self.footprint = tile, footprint
        self.accum = None    # densify statistic (summed screen-space position-gradient norms), when tracked
        self.vis = None      # steps in which each Gaussian touched a tile
        # Adam step count and the step's constants on the device (fused path), so steps can be graph-replayed
        self.adam_state = torch.zeros(4, dtype=torch.int32, device=device)
        self.graphs = None
        self._pending = None     # (camera bytes, frame, its projection generation): a projection already made
        self._graph_next = None  # per captured graph: the view whose projection it leaves behind (chained capture)

    def state_dict(self):
        """The training state as host tensors, for a checkpoint: the parameters
        (means_sigma with log sigma, logit opacity, colour), the Adam moments,
        the step count (host and device copies), the densify statistic when it
        is tracked, and the settings a resumed run needs. Captured graphs are not
        part of it (capture again after resuming)."""
        host = lambda ts: [t.detach().cpu().clone() for t in ts]  # noqa: E731
        ms, op, col = host(self._views(self.flat))
        d = {"means_sigma": ms, "opacity": op, "color": col, "m": host(self.m_views), "v": host(self.v_views),
             "t": int(self.t), "adam_state": self.adam_state.cpu().clone(), "sh_degree": int(self.sh_degree),
             "tile": int(self.tile), "lr": float(self.lr), "fused": bool(self.fused),
             "footprint": int(self.footprint), "ssim_lambda": float(self.ssim_lambda)}
        if self.accum is not None:
            d["accum"], d["vis"] = self.accum.cpu().clone(), self.vis.cpu().clone()
        return d

    @classmethod
    def from_state_dict(cls, d, device="cuda"):
        """A TrainStep that continues from a state_dict(): the next step is the
        one that followed the checkpoint. Entry capacities are not stored, so the
        first step of each view runs with check=True."""
        ts = cls(d["means_sigma"].to(device), d["opacity"].to(device), d["color"].to(device), d["sh_degree"],
                 tile=d["tile"], lr=d["lr"], device=device, fused=d["fused"], footprint=d["footprint"],
                 ssim_lambda=d["ssim_lambda"])
        for dst, src in zip(ts.m_views + ts.v_views, list(d["m"]) + list(d["v"])):
            dst.copy_(src)
        ts.t = int(d["t"])
        ts.adam_state.copy_(d["adam_state"])
        if "accum" in d:
            ts.accum, ts.vis = d["accum"].to(device), d["vis"].to(device)
        return ts

    def save(self, path):
        """Write state_dict() to `path` (torch.save)."""
        torch.save(self.state_dict(), path)

    @classmethod
    def load(cls, path, device="cuda"):
        """from_state_dict of a file written by save()."""
        return cls.from_state_dict(torch.load(path, map_location="cpu"), device)

    def _views(self, flat):
        n, C = self.n, self.C
        return (flat[:4 * n].view(n, 4), flat[self.o_op:self.o_op + n], flat[self.o_col:self.o_col + C * n].view(n, C))

    def _projected(self, c, frame):
        """Whether `frame` already holds this scene's projection for camera c
        (left there by the previous step's fused pass, and not touched since)."""
        p = self._pending
        return (p is not None and p[0] == bytes(c) and p[1] is frame and p[2] == getattr(frame, "proj_gen", 0)
                and frame.n == self.n)

    def _mark_projected(self, c, frame):
        frame.proj_gen = getattr(frame, "proj_gen", 0) + 1
        self._pending = (bytes(c), frame, frame.proj_gen)

    def _side(self):
        """The stream the step's host copies run on (created once)."""
        if getattr(self, "_side_stream", None) is None:
            self._side_stream = torch.cuda.Stream(device=self.flat.device)
        return self._side_stream

    def step(self, cam, target, check=False, stream=None, marks=None, next_cam=None, target_host=None,
             loss_host=None):
        """One training step on `stream`. `marks`, if given, is called with a
        stage name after each stage is enqueued (the benchmark records CUDA
        events there). With next_cam (fused path), the step's last pass also
        projects the updated scene for next_cam, and the next step on that
        camera starts at the binning (the projection arrays of the returned
        frame then hold next_cam's view when it has the same size).
        target_host (pinned host tensor): copied into `target` by the step itself,
        on a side stream that overlaps the binning and the forward and joins
        before the loss; loss_host (pinned, one float): the loss is copied there
        on the side stream while the backward runs, joined at the step's end.
        Both become part of a captured graph."""
        c = cam if isinstance(cam, igs.IgsCamera) else igs.camera(cam)
        cur = stream if stream is not None else torch.cuda.current_stream(self.flat.device)
        side = self._side() if (target_host is not None or loss_host is not None) else None
        if target_host is not None:
            side.wait_stream(cur)  # every earlier reader of `target` is done
            with torch.cuda.stream(side):
                target.copy_(target_host, non_blocking=True)
        key = (c.width, c.height)
        if key not in self._img:
            self._img[key] = torch.empty((3, c.height, c.width), dtype=torch.float32, device=self.flat.device)
            self._dimg[key] = torch.empty_like(self._img[key])
        img, dimg = self._img[key], self._dimg[key]
        r = self.renderer
        mark = marks or (lambda name: None)
        if check:
            img, frame = r.run_forward(self.scene, c, img=img, check=True, stream=stream)
        else:
            frame = r.frame(self.scene.n, c, r.capacity_for(self.scene.n, c))
            if not self._projected(c, frame):
                igs.project(self.scene, c, r.opts, frame, stream)
                frame.proj_gen = getattr(frame, "proj_gen", 0) + 1
            mark("project")
            igs.bin_sort(frame, r.opts, stream)
            mark("bin_sort")
            igs.render_fwd_clear(frame, r.opts, img, self.g2d, stream)  # clears g2d for the adjoint below
        mark("blend_fwd")
        if target_host is not None:
            cur.wait_stream(side)  # the target has arrived
        if self.ssim_lambda > 0.0:
            if key not in self._work:
                self._work[key] = torch.empty(igs.ssim_work_bytes(3, c.height, c.width) // 4, dtype=torch.float32,
                                              device=self.flat.device)
            igs.l1_ssim_loss(img, target, self.ssim_lambda, self.loss, dimg, self._work[key], stream=stream)
            mark("l1_ssim")
        else:
            igs.l1_loss(img, target, self.loss, dimg, stream)
            mark("l1")
        if loss_host is not None:
            side.wait_stream(cur)  # the loss is final
            with torch.cuda.stream(side):
                loss_host.copy_(self.loss, non_blocking=True)
        if check:
            igs.blend_bwd(frame, r.opts, dimg, self.g2d, stream)
        else:
            igs.blend_bwd_acc(frame, r.opts, dimg, self.g2d, stream)
        mark("blend_bwd")
        if self.accum is not None:
            igs.grad_accum(self.g2d, frame.count(), self.accum, self.vis, stream)
        self.t += 1
        self._pending = None
        if self.fused and next_cam is not None:
            nc = next_cam if isinstance(next_cam, igs.IgsCamera) else igs.camera(next_cam)
            nframe = r.frame(self.scene.n, nc, r.capacity_for(self.scene.n, nc))
            igs.project_bwd_adam_next(self.scene, c, r.opts, frame, self.g2d, self.m_views, self.v_views,
                                      self.adam_state, nc, nframe, lr=self.lr, stream=stream)
            self._mark_projected(nc, nframe)
            mark("project_bwd_adam")
        elif self.fused:
            igs.project_bwd_adam_dev(self.scene, c, r.opts, frame, self.g2d, self.m_views, self.v_views,
                                     self.adam_state, lr=self.lr, stream=stream)
            mark("project_bwd_adam")
        else:
            igs.project_bwd(self.scene, c, r.opts, frame, self.g2d, self.g_ms, self.g_op, self.g_col, stream)
            mark("project_bwd")
            igs.adam(self.flat, self.grad, self.m, self.v, self.t, lr=self.lr, stream=stream)
            mark("adam")
        if loss_host is not None:
            cur.wait_stream(side)  # the loss copy joins the step
        return frame

    def capture(self, cams, targets, chain=False, targets_host=None, losses_host=None):
        """Record one training step per (camera, target) into its own CUDA graph
        (fused path: the Adam step count lives on the device, so replays keep
        counting). Each view must have run once with check=True before (its entry
        capacity is then known). Replay with replay(k); the graphs read the
        `targets` tensors as they are at replay time. With chain=True, graph k
        ends by projecting view k + 1 (cyclically) and starts at its binning:
        replays in the order 0, 1, 2, ... skip every projection pass; replay(k)
        after anything else first projects view k on the current stream. With
        targets_host / losses_host (pinned host tensors, one per view), each
        graph also copies its target in from the host and its loss out to the
        host (step's target_host / loss_host)."""
        if not self.fused:
            raise RuntimeError("graph capture needs the fused projection backward + Adam")
        t0 = self.t
        cams = [c if isinstance(c, igs.IgsCamera) else igs.camera(c) for c in cams]
        V = len(cams)
        r = self.renderer
        cur = torch.cuda.current_stream()
        s = torch.cuda.Stream(device=self.flat.device)
        s.wait_stream(cur)
        graphs, frames, nexts = [], [], []
        with torch.cuda.stream(s):
            for k, (c, tgt) in enumerate(zip(cams, targets)):
                frame = r.frame(self.scene.n, c, r.capacity_for(self.scene.n, c))
                if chain:  # recorded as if the previous graph had projected this view
                    self._mark_projected(c, frame)
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s):
                    self.step(c, tgt, stream=s, next_cam=cams[(k + 1) % V] if chain else None,
                              target_host=targets_host[k] if targets_host is not None else None,
                              loss_host=losses_host[k] if losses_host is not None else None)
                graphs.append(g)
                frames.append(frame)
                nexts.append((k + 1) % V if chain else None)
        cur.wait_stream(s)
        self.t = t0  # recording ran nothing
        self._pending = None
        self.graphs = graphs
        self._graph_cams, self._graph_frames, self._graph_next = cams, frames, nexts
        return graphs

    def replay(self, k):
        """Replay the captured step of view k on the current stream."""
        if self._graph_next[k] is not None:  # chained graph: it starts at the binning
            c, frame = self._graph_cams[k], self._graph_frames[k]
            if not self._projected(c, frame):
                igs.project(self.scene, c, self.renderer.opts, frame)
                frame.proj_gen = getattr(frame, "proj_gen", 0) + 1
            self.graphs[k].replay()
            j = self._graph_next[k]
            self._mark_projected(self._graph_cams[j], self._graph_frames[j])
        else:
            self.graphs[k].replay()
            self._pending = None
        self.t += 1

    def track_grad_norm(self):
        """Start (or restart) the densify statistic: every later step adds each
        visible Gaussian's screen-space position-gradient norm to accum and one
        to vis."""
        self.accum = torch.zeros(self.n, dtype=torch.float32, device=self.flat.device)
        self.vis = torch.zeros(self.n, dtype=torch.int32, device=self.flat.device)

    def densify(self, op_min, tau_g, scale_min, capacity):
        """Delete Gaussians whose stored opacity logit is below op_min, divide those
        whose mean screen-space gradient norm since track_grad_norm() exceeds tau_g
        (and whose log sigma >= scale_min) into eight half-scale children, within
        `capacity` Gaussians (libigs's igs_densify); parameters and Adam moments
        move to new flat buffers. Reads the new count back (one synchronisation);
        the Adam step count continues. The next step of each view should run with
        check=True (the entry capacity of the new scene is not known yet)."""
        if self.accum is None:
            raise RuntimeError("densify needs track_grad_norm() first")
        dev = self.flat.device
        cap = int(capacity)
        C = self.C
        outs = [(torch.empty((cap, 4), device=dev), torch.empty(cap, device=dev), torch.empty((cap, C), device=dev))
                for _ in range(3)]
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        work = torch.empty(igs.densify_work_bytes(self.n), dtype=torch.uint8, device=dev)
        igs.densify(self.scene, self.m_views, self.v_views, self.sh_degree, 1, self.accum, self.vis, op_min, tau_g,
                    scale_min, outs[0], outs[1], outs[2], count, work)
        k = int(count.item())
        self._relayout(k, outs)
        self.track_grad_norm()
        return k

    def merge(self, lo, cell, scale_max):
        """Merge the eligible Gaussians (log sigma <= scale_max, finite mean,
        opacity logit >= -41.58883, i.e. opacity >= 2^-60) that share a grid cell of side `cell` from the corner lo
        into one each (libigs's igs_merge: opacity-weighted mean and colour,
        moment-matched scale, opacity 1 - prod (1 - o_k) capped at 0.99, zero
        moments); parameters and Adam moments move to new flat buffers. Reads the
        new count back (one synchronisation); the Adam step count continues."""
        dev = self.flat.device
        n, C = self.n, self.C
        outs = [(torch.empty((max(n, 1), 4), device=dev), torch.empty(max(n, 1), device=dev),
                 torch.empty((max(n, 1), C), device=dev)) for _ in range(3)]
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        work = torch.empty(igs.merge_work_bytes(n), dtype=torch.uint8, device=dev)
        igs.merge(self.scene, self.m_views, self.v_views, self.sh_degree, 1, lo, cell, scale_max, outs[0], outs[1],
                  outs[2], count, work)
        k = int(count.item())
        if k < 0:
            raise igs.IgsError(igs.ERR_DEVICE_TIMEOUT, "merge: the device sort gave up on a bounded wait")
        self._relayout(k, outs)
        if self.accum is not None:
            self.track_grad_norm()
        return k

    def _relayout(self, n, arrays):
        """New flat buffers for n Gaussians, filled from (params, m, v) arrays."""
        self.n = n
        a = lambda x: (x + 63) // 64 * 64  # noqa: E731
        self.o_op = a(4 * n)
        self.o_col = a(self.o_op + n)
        size = a(self.o_col + self.C * n)
        dev = self.flat.device
        self.flat = torch.zeros(size, dtype=torch.float32, device=dev)
        self.grad = torch.zeros_like(self.flat)
        self.m = torch.zeros_like(self.flat)
        self.v = torch.zeros_like(self.flat)
        for flat, (ms, op, col) in zip((self.flat, self.m, self.v), arrays):
            a_ms, a_op, a_col = self._views(flat)
            a_ms.copy_(ms[:n])
            a_op.copy_(op[:n])
            a_col.copy_(col[:n])
        self.ms, self.op, self.col = self._views(self.flat)
        self.g_ms, self.g_op, self.g_col = self._views(self.grad)
        self.m_views = self._views(self.m)
        self.v_views = self._views(self.v)
        self.scene = igs.Scene(self.ms, self.op, self.col)
        self.g2d = torch.empty((n, 8), dtype=torch.float32, device=dev)
        self.graphs = None  # captured steps refer to the old buffers
        self._pending = None
