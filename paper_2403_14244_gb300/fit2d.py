"""The paper's 2D experiment (Sec. 3): fit an image with a sum of isotropic
kernels, initialised by a QuadTree (Sec. 3.1) and optimised by back-propagation
of the loss (1 - lambda) L1 + lambda (1 - SSIM).

Every step runs in libigs's kernels (``igs.fit2d_render``, ``igs.l1_ssim_loss``,
``igs.fit2d_backward``, ``igs.fit2d_adam``); ``Fit2D.capture`` records
``inner`` iterations into one CUDA graph (the Adam step count lives on the
device, so a replay continues the optimisation), and ``run`` replays it."""
from __future__ import annotations

import torch

from . import igs

# Adam learning rates per particle slot (mu_x, mu_y, log sigma, A_r, A_g, A_b, -, -):
# pixels, log units and colour units per step.
DEFAULT_LR = (0.2, 0.2, 0.02, 0.02, 0.02, 0.02, 0.0, 0.0)


class Fit2D:
    """Fitting state for one RGB target image ([3][S][S] on the GPU, S a power
    of two <= 512): QuadTree particles (at most k_max, cells >= min_cell wide),
    support D (pixels), loss weight lam."""

    def __init__(self, target, k_max, D, min_cell=3, lam=0.2, lr=DEFAULT_LR, device="cuda"):
        if target.dim() != 3 or target.shape[0] != 3 or target.shape[1] != target.shape[2]:
            raise ValueError("target must be [3][S][S]")
        self.target = target.contiguous()
        self.D, self.lam, self.lr = float(D), float(lam), tuple(float(x) for x in lr)
        S = target.shape[1]
        self.side = S
        buf = torch.zeros((k_max, 8), dtype=torch.float32, device=device)
        count = torch.zeros(1, dtype=torch.int32, device=device)
        work = torch.empty(igs.quadtree_work_bytes(S, min_cell), dtype=torch.uint8, device=device)
        igs.quadtree_init(self.target, k_max, min_cell, buf, count, work)
        self.k = int(count.item())   # one synchronisation, at set-up
        self.particles = buf[:self.k].clone()
        self.initial = self.particles.clone()
        self.grad = torch.zeros_like(self.particles)
        self.m = torch.zeros_like(self.particles)
        self.v = torch.zeros_like(self.particles)
        self.state = torch.zeros(2, dtype=torch.int32, device=device)
        self.img = torch.empty_like(self.target)
        self.dimg = torch.empty_like(self.target)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.ssim = torch.zeros(1, dtype=torch.float32, device=device)
        self.work = torch.empty(igs.ssim_work_bytes(3, S, S) // 4, dtype=torch.float32, device=device)
        self.graph = None
        self.inner = 0
        self.accum = None       # summed position-gradient norms (densify statistic), when tracked
        self.accum_iters = 0    # iterations summed into accum

    def render(self, stream=None):
        igs.fit2d_render(self.particles, self.D, self.img, stream)
        return self.img

    def step(self, stream=None):
        """One iteration: render, loss and its image gradient, particle gradient, Adam."""
        igs.fit2d_render(self.particles, self.D, self.img, stream)
        igs.l1_ssim_loss(self.img, self.target, self.lam, self.loss, self.dimg, self.work, ssim=self.ssim,
                         stream=stream)
        igs.fit2d_backward(self.particles, self.D, self.dimg, self.grad, stream)
        if self.accum is not None:
            igs.fit2d_grad_accum(self.grad, self.accum, stream)
            self.accum_iters += 1
        igs.fit2d_adam(self.particles, self.grad, self.m, self.v, self.lr, self.state, stream=stream)

    def track_grad_norm(self):
        """Start summing each particle's position-gradient norm (the statistic
        densify() divides by); drops a captured graph, which did not sum it."""
        self.accum = torch.zeros(self.k, dtype=torch.float32, device=self.particles.device)
        self.accum_iters = 0
        self.graph = None

    def densify(self, tau_a, tau_g, log_sigma_min, capacity):
        """Delete particles with max |A| < tau_a, divide those whose mean
        position-gradient norm since the last densify exceeds tau_g (and whose
        log sigma >= log_sigma_min) into four half-scale children, within
        `capacity` particles (libigs's igs_fit2d_densify). Reads the new count
        back (one synchronisation) and drops the captured graph."""
        if self.accum is None or self.accum_iters == 0:
            raise RuntimeError("densify needs track_grad_norm() and at least one step")
        dev = self.particles.device
        out = torch.empty((capacity, 8), dtype=torch.float32, device=dev)
        om, ov = torch.empty_like(out), torch.empty_like(out)
        count = torch.zeros(1, dtype=torch.int32, device=dev)
        igs.fit2d_densify(self.particles, self.m, self.v, self.accum, self.accum_iters, tau_a, tau_g, log_sigma_min,
                          out, om, ov, count)
        k = int(count.item())
        self.particles, self.m, self.v = out[:k].clone(), om[:k].clone(), ov[:k].clone()
        self.k = k
        self.grad = torch.zeros_like(self.particles)
        self.track_grad_norm()
        return k

    def capture(self, inner=10):
        """Record `inner` iterations into one CUDA graph (after one eager step,
        which also loads the kernels)."""
        self.step()
        torch.cuda.synchronize()
        iters0 = self.accum_iters
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                for _ in range(inner):
                    self.step()
        torch.cuda.current_stream().wait_stream(s)
        self.accum_iters = iters0       # recording ran nothing
        self.graph, self.inner = g, inner
        return g

    def run(self, iters):
        """Replay the captured graph until at least `iters` further iterations ran."""
        if self.graph is None:
            self.capture()
        n = 0
        while n < iters:
            self.graph.replay()
            n += self.inner
            if self.accum is not None:
                self.accum_iters += self.inner
        return n

    def steps_done(self):
        return int(self.state[0].item())
