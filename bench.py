"""Benchmark of the isotropic Gaussian splatting hot path on GB300.

Workload (one GPU): the training step of a 3M-Gaussian scene (means U[-1,1]^3,
sigma log-uniform [0.005, 0.05] stored as log sigma, opacity U[0.05, 0.95]
stored as a logit, degree-3 SH with DC from U[0,1] RGB), 1297x840 images, 16
cameras on a ring of radius 4. One step = one view: project, bin + sort,
forward blend, L1 loss against that view's seeded target, backward blend,
projection backward, Adam over all 53 parameters of every Gaussian. Steps cycle
through the 16 views. All inputs are synthetic and seeded; they live in HBM
before the timed region; the per-step working set (parameters, Adam state,
gradients: 2.5 GB) is far larger than L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0). --impl reference times the CPU oracle (the
reference arm of this method: the paper ships no code) on the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "1080p frames/s & fwd+bwd steps/s at 3M isotropic Gaussians; serve p50/p99 ms"
WORKLOAD = "train_step_3M_sh3_1297x840_ring16"
STAGES_L1 = ("project", "bin_sort", "blend_fwd", "l1", "blend_bwd", "project_bwd_adam")
STAGES_SSIM = ("project", "bin_sort", "blend_fwd", "l1_ssim", "blend_bwd", "project_bwd_adam")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("mine", "reference"), default="mine")
    ap.add_argument("--n", type=int, default=3_000_000, help="Gaussians (default: the 3M workload)")
    ap.add_argument("--no-extra", action="store_true", help="skip the 1080p forward / fwd+bwd lines")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--tile", type=int, default=32, choices=(8, 16, 32),
                    help="binning tile edge in pixels (the blends run per 8 x 8 block of it)")
    ap.add_argument("--footprint", type=int, default=0, choices=(0, 1),
                    help="tiles of a Gaussian: 0 its bounding rectangle, 1 the tiles its disc meets")
    ap.add_argument("--ssim", type=float, default=0.0,
                    help="lambda of the loss (1 - lambda) L1 + lambda (1 - SSIM) in the timed step (0: L1)")
    ap.add_argument("--only", choices=("merge", "batched"), default=None,
                    help="measure one side line alone (no training step, no JSON contract): merge on the training "
                         "scene, or batched: one batched render of --batch-views sphere views of a --batch-n RGB "
                         "scene at 32-pixel tiles and 64-entry staging (the autotuned setting of the batched line), "
                         "captured once and replayed --steps times after --warmup replays")
    ap.add_argument("--batch-n", type=int, default=2_000_000, help="Gaussians of the --only batched scene")
    ap.add_argument("--batch-views", type=int, default=32, help="views of the --only batched render")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device):
    """The largest value of x over the ranks (the slowest rank's time); x itself
    when one process runs. Every rank must call it (a collective)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units of all ranks (each does the same work: weak scaling) per second of
    the slowest rank."""
    return world * units_per_rank / seconds


# GB300's stated HBM3e bandwidth (8 stacks at 3996 MHz): the figure a copy-based
# measurement stays below; fractions are reported against both.
HBM_NOMINAL_GBS = 7900.0


def load_peaks():
    """HBM peak for the rooflines: the measured copy bandwidth (a torch
    b.copy_ over 2 GiB, read + write bytes) when the pool's measurement file is
    there, else the fallback figure of an earlier GB300 measurement."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured copy (torch b.copy_, read + write bytes)"
    except Exception:
        return 6800.0, "fallback (an earlier GB300 copy measurement)"


def stage_rooflines(stage_ms, n, C, P, M, tiles, peak_hbm):
    """Algorithmic bytes per launch of every stage (per-unit figures in the
    comments of `model`, times the units of one step) and the bandwidth they
    imply over the stage's measured time. The blends are
    bound by issue slots, not HBM: their bytes (entry gathers, per-pixel buffers)
    are listed for context."""
    params = 5 + C
    model = {
        # read means_sigma, opacity, colour; write record, rectangle, count, depth key
        "project": ("hbm", n * (16 + 4 + 4 * C) + n * (32 + 8 + 4 + 4)),
        # lower bound of the binning: depth keys, rectangles, counts in; order, entries, ranges out
        "bin_sort": ("hbm", n * (4 + 8 + 4) + n * 4 + 4 * M + 8 * tiles),
        # per entry: id + 32-byte record; per pixel: image, T_final, n_contrib
        "blend_fwd": ("alu", M * (4 + 32) + P * (12 + 4 + 4)),
        "l1": ("hbm", P * 3 * 4 * 3),
        # per entry: img, target in and three partial maps out; maps, img, target in and gradient out
        "l1_ssim": ("hbm", P * 3 * 44),
        # per entry: id + record; per pixel: dL, T_final, n_contrib; per Gaussian: 2D gradient
        "blend_bwd": ("alu", M * (4 + 32) + P * (12 + 4 + 4) + n * 32),
        # read params, 2D gradient, count, m, v; write params, m, v
        "project_bwd_adam": ("hbm", n * (4 * params + 32 + 4 + 8 * params) + n * 12 * params),
        # the same, and the next view's record, rectangle, count and depth key written
        "project_bwd_adam_next": ("hbm", n * (4 * params + 32 + 4 + 8 * params) + n * 12 * params
                                  + n * (32 + 8 + 4 + 4)),
    }
    total = sum(stage_ms.values())
    out = []
    for s, ms in stage_ms.items():
        bound, nbytes = model[s]
        gbs = nbytes / (ms / 1e3) / 1e9
        row = {"stage": s, "ms": round(ms, 4), "share": round(ms / total, 4), "bound": bound, "bytes": int(nbytes)}
        if bound == "hbm":
            row.update({"achieved": round(gbs, 1), "frac": round(gbs / peak_hbm, 4),
                        "frac_nominal": round(gbs / HBM_NOMINAL_GBS, 4)})
        else:  # issue-bound: the bytes (mostly L2 gathers) are context, not a roofline
            row.update({"bytes_per_s_context": round(gbs, 1), "frac": None})
        out.append(row)
    return out


# ncu counters per launch, from profiles/*.json, valid only while the kernel's
# sources hash to the value recorded with the capture.
TRAFFIC_SOURCES = {
    "project_bwd_adam": ("project.cu", "projection.cuh", "common.cuh"),
    "project_bwd_adam_next": ("project.cu", "projection.cuh", "common.cuh"),
    "project": ("project.cu", "projection.cuh", "common.cuh"),
    "l1": ("train.cu", "common.cuh"),
    "blend_fwd": ("blend.cu", "blendtile.cuh", "common.cuh"),
    "blend_bwd": ("blend.cu", "blendtile.cuh", "warp.cuh", "common.cuh"),
}


def sources_sha(stage):
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES[stage]:
        with open(os.path.join(ROOT, "paper_2403_14244_gb300", "csrc", name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def _counter_rows(name):
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            return json.load(f)["rows"]
    except (OSError, ValueError, KeyError):
        return []


def traffic_per_launch(stage, n):
    """dram__bytes_read.sum + dram__bytes_write.sum of one launch of the stage's
    kernel (profiles/dram_traffic.json), scaled from the captured size to n
    Gaussians; None when no capture matches the current sources."""
    if stage not in TRAFFIC_SOURCES:
        return None
    sha = sources_sha(stage)
    for row in _counter_rows("dram_traffic.json"):
        if row.get("stage") == stage and row.get("sources_sha16") == sha:
            return int(float(row["bytes"]) * n / float(row["n_captured"]))
    return None


def issue_per_launch(stage, workload):
    """Warp instructions issued per launch (smsp__inst_executed.sum, mean over
    the captured launches: consecutive views of the workload) from
    profiles/issue_counts.json; None when no capture matches the sources."""
    if stage not in TRAFFIC_SOURCES:
        return None
    sha = sources_sha(stage)
    for row in _counter_rows("issue_counts.json"):
        if row.get("stage") == stage and row.get("sources_sha16") == sha and row.get("workload") == workload:
            return float(row["warp_inst_per_launch"])
    return None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.out = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={device_index}", "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------- GPU arm --------

def build_workload(n, device, footprint=0, tile=32):
    import numpy as np
    import torch

    from paper_2403_14244_gb300 import igs, scenes
    from paper_2403_14244_gb300.render import TrainStep

    sc, cams = scenes.workload_train_3m(n=n)
    ts = TrainStep(torch.from_numpy(sc.means_sigma).to(device), torch.from_numpy(sc.opacity).to(device),
                   torch.from_numpy(sc.color).to(device), sh_degree=3, tile=tile, lr=1e-3, device=device,
                   footprint=footprint)
    targets_host = [torch.from_numpy(scenes.train_target(k)).pin_memory() for k in range(len(cams))]
    targets = [t.to(device) for t in targets_host]
    cam_s = [igs.camera(c) for c in cams]
    return sc, cams, cam_s, ts, targets, targets_host, np


E2E_MIN_STEPS = 400
E2E_WARMUP = 16


def workload_config(args, n, world):
    """The `config` of both arms' JSON lines (the same workload either way)."""
    return {"workload": WORKLOAD, "n_gaussians": n, "sh_degree": 3, "image": [1297, 840], "views": 16,
            "tile": args.tile, "footprint": "rectangle" if args.footprint == 0 else "disc rows",
            "optimizer": "adam lr 1e-3", "params": "mu, log sigma, logit o, SH",
            "loss": "l1" if args.ssim == 0 else f"(1 - {args.ssim}) l1 + {args.ssim} (1 - ssim)",
            "l2": "no flush: per-step working set 2.5 GB > 129 MB L2",
            "parallelism": f"replicas x{world} (no collective)"}


def run_e2e(ts, cam_s, targets, targets_host, dev, V, warm, steps, barrier, world):
    """Seconds (max over ranks) for `steps` end-to-end steps after `warm` untimed
    ones. Each step's graph copies its target in from pinned host memory (on a
    side stream that overlaps the step's binning and forward) and its loss out to
    pinned host memory (overlapping the backward): TrainStep.capture with
    targets_host / losses_host, the public API's way to train from host data."""
    import torch

    losses_host = [torch.empty(1, dtype=torch.float32).pin_memory() for _ in range(V)]
    ts.capture(cam_s, targets, chain=True, targets_host=targets_host, losses_host=losses_host)

    def run(count):
        for k in range(count):
            ts.replay(k % V)

    run(warm)
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    run(steps)
    torch.cuda.synchronize(dev)
    seconds = time.perf_counter() - t0
    assert all(bool(torch.isfinite(x).all()) for x in losses_host), "a step's loss did not reach the host"
    return max_over_ranks(seconds, world, dev)


def issue_rooflines(stages, sms, sm_mhz):
    """The blends are bound by instruction issue: each SM's 4 schedulers issue at
    most one warp instruction per clock. Where profiles/issue_counts.json holds
    the warp instructions per launch for the current sources, the stage gets
    achieved = instructions / mean stage time and frac of sms * 4 * clock
    (the median SM clock sampled during the timed region)."""
    if not sm_mhz:
        return
    peak = sms * 4 * sm_mhz * 1e6
    for r in stages:
        if r["bound"] != "alu":
            continue
        inst = issue_per_launch(r["stage"], WORKLOAD)
        if inst is None:
            continue
        achieved = inst / (r["ms"] / 1e3)
        r.update({"warp_inst_per_launch": int(inst), "achieved": round(achieved / 1e12, 4),
                  "peak": round(peak / 1e12, 4), "unit": "T warp-instructions/s", "frac": round(achieved / peak, 4)})


def run_mine(args, world, rank, local):
    import torch

    from paper_2403_14244_gb300 import igs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    igs.load()
    sc, cams, cam_s, ts, targets, targets_host, np = build_workload(args.n, dev, args.footprint, args.tile)
    ts.ssim_lambda = args.ssim
    STAGES = STAGES_L1 if args.ssim == 0 else STAGES_SSIM
    V = len(cams)
    stream = torch.cuda.current_stream(dev)
    # capacity calibration: every view once with a status check (untimed set-up)
    for k in range(V):
        ts.step(cam_s[k], targets[k], check=True)
    # every step ends by projecting the next view (views in cyclic order), so the
    # next step starts at its binning
    for k in range(args.warmup):
        ts.step(cam_s[k % V], targets[k % V], next_cam=cam_s[(k + 1) % V])
    torch.cuda.synchronize(dev)
    # per-stage times: eager steps with CUDA events between the stages (untimed for the headline)
    stage_steps = min(args.steps, 128)
    stage_ev = []
    for k in range(args.warmup, args.warmup + stage_steps):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)]
        evs[0].record(stream)
        it = iter(evs[1:])
        ts.step(cam_s[k % V], targets[k % V], marks=lambda name, it=it: next(it).record(stream),
                next_cam=cam_s[(k + 1) % V])
        stage_ev.append(evs)
    torch.cuda.synchronize(dev)
    stage_ms = {s: 0.0 for s in STAGES}
    for evs in stage_ev:
        for i, s in enumerate(STAGES):
            stage_ms[s] += evs[i].elapsed_time(evs[i + 1])
    stage_ms = {s: v / stage_steps for s, v in stage_ms.items()}
    # the projection ran inside the previous step's last pass: its own interval is empty
    stage_ms.pop("project")
    stage_ms["project_bwd_adam_next"] = stage_ms.pop("project_bwd_adam")
    eager_ms = sum(stage_ms.values())
    # one CUDA graph per view's step (the Adam step count lives on the device), chained:
    # graph k ends by projecting view k + 1
    launches0 = igs.launch_count()
    ts.capture(cam_s, targets, chain=True)
    launches_per_step = (igs.launch_count() - launches0) / V
    for k in range(V):
        ts.replay(k)
    torch.cuda.synchronize(dev)

    # -------- timed region: K steps (graph replays), device time on the launching stream
    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    clocks = ClockSampler(local)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize(dev)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        ts.replay(k % V)
    end.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    launches = launches_per_step * args.steps
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(start.elapsed_time(end), world, dev)
    # the entry capacity used in the timed region held for every view: re-run
    # each view's binning at that capacity (untimed) and read its status
    entries = []
    for k in range(V):
        _, f = ts.renderer.run_forward(ts.scene, cam_s[k], check=False)
        st, info = igs.frame_status(f)
        assert st == igs.OK, f"view {k}: device status {st} after the timed region"
        entries.append(int(info[0]))
    tiles = f.tiles
    ms_per_step = elapsed_ms / args.steps
    value = whole_job_rate(args.steps, world, elapsed_ms / 1e3)

    # -------- end to end: host target in pinned memory -> device, step, loss -> host, every step,
    # inside the step's own graph (the target's copy overlaps the binning and the forward, the
    # loss's the backward). A fixed window (at least E2E_MIN_STEPS steps, after E2E_WARMUP untimed
    # ones) whatever --steps is, so that start-up costs do not decide the number. The graphs are
    # captured again for this (the timed region above replays graphs without the copies).
    e2e_steps = max(args.steps, E2E_MIN_STEPS)
    e2e_s = run_e2e(ts, cam_s, targets, targets_host, dev, V, E2E_WARMUP, e2e_steps, barrier, world)
    e2e = {"value": round(whole_job_rate(e2e_steps, world, e2e_s), 3), "unit": "steps/s",
           "h2d_bytes_per_step": int(targets[0].numel() * 4), "d2h_bytes_per_step": 4, "steps": e2e_steps,
           "overlap": "each step's graph copies its target from pinned host memory on a side stream during "
                      "its binning and forward, and its loss to pinned host memory during its backward"}

    # -------- rooflines: every stage against its bound, headline = largest HBM-bound stage
    peak_hbm, peak_kind = load_peaks()
    n, C = ts.n, ts.C
    P = cams[0].width * cams[0].height
    M = sum(entries) / len(entries)
    stages = stage_rooflines(stage_ms, n, C, P, M, tiles, peak_hbm)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_rooflines(stages, sms, clk.get("sm_mhz"))
    hbm = [r for r in stages if r["bound"] == "hbm"]
    top = max(hbm, key=lambda r: r["ms"])
    roofline = {"kernel": top["stage"], "bound": "hbm", "achieved": top["achieved"], "peak": peak_hbm,
                "unit": "GB/s", "frac": top["frac"], "traffic": traffic_per_launch(top["stage"], n),
                "peak_kind": peak_kind, "peak_nominal": HBM_NOMINAL_GBS, "frac_nominal": top["frac_nominal"],
                "share_of_step": top["share"]}
    if top["frac"] > 1.0:
        roofline["note"] = ("frac > 1: the kernel moves its algorithmic bytes faster than the measured copy "
                            "baseline; against the nominal HBM peak it is frac_nominal")
    dominant = max(stages, key=lambda r: r["ms"])
    binrow = next(r for r in stages if r["stage"] == "bin_sort")
    binning = {"ms": binrow["ms"], "bytes": binrow["bytes"], "achieved_gbs": binrow["achieved"],
               "frac": binrow["frac"], "frac_nominal": binrow["frac_nominal"], "target_frac_nominal": 0.6,
               "met": binrow["frac_nominal"] >= 0.6,
               "bytes_model": "20 B per Gaussian (depth key, rectangle, count in; order out) + 4 B per entry "
                              "+ 8 B per tile"}

    extra = {}
    if not args.no_extra and args.ssim == 0:
        extra["train_step_l1_ssim"] = run_ssim_steps(ts, cam_s, targets, stream, dev, min(args.steps, 100),
                                                     peak_hbm)
    if not args.no_extra:
        extra["densify_3M"] = run_densify3d(ts, cam_s, targets, stream, dev, peak_hbm)
        extra["merge_3M"] = run_merge3d(ts, stream, dev, peak_hbm)
        extra.update(run_extra(dev, np, args.tile))

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generators, no dataset)",
        "config": workload_config(args, n, world),
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        "graph": "one CUDA graph per view's step, replayed (the Adam step count on the device)",
        "eager_ms_per_step": round(eager_ms, 4),
        "stage_ms": {s: round(v, 4) for s, v in stage_ms.items()},
        "roofline": roofline, "dominant": {"stage": dominant["stage"], "bound": dominant["bound"],
                                           "share_of_step": dominant["share"]},
        "stages": stages, "binning": binning, "entries_mean": round(M), "extra": extra,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(sc, cams, args.cpu_budget, args.ssim)
        if not args.no_extra:
            extra["cpu_oracle_small_configs"] = cpu_configs()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_densify3d(ts, cam_s, targets, stream, dev, peak_hbm, steps=32, reps=3):
    """Densify / prune of the training scene: the cost of the per-step statistic
    (steps/s with and without it), and one keep / delete / divide pass
    (igs_densify) over all Gaussians after `steps` tracked steps: delete opacity
    below 0.005, divide the Gaussians whose mean screen-space gradient norm is in
    the top tenth of those with a non-zero gradient (threshold read on the host)
    and whose sigma >= 0.01, capacity
    2n. Bandwidth over the pass's algorithmic bytes: 28 B per Gaussian twice
    (flags: opacity, statistic, scale), 2 x 636 B per kept Gaussian (parameters
    and moments read and written), 212 + 8 x 636 B per divided one."""
    import math

    import numpy as np
    import torch

    from paper_2403_14244_gb300 import igs

    V = len(cam_s)

    def timed(n_steps):
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for k in range(n_steps):
            ts.step(cam_s[k % V], targets[k % V], next_cam=cam_s[(k + 1) % V])
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / n_steps

    plain_ms = timed(steps)
    ts.track_grad_norm()
    tracked_ms = timed(steps)
    n, C = ts.n, ts.C
    acc, vis = ts.accum.cpu().numpy(), ts.vis.cpu().numpy().view(np.uint32)
    moved = (vis > 0) & (acc > 0)
    tau_g = float(np.quantile(acc[moved] / vis[moved], 0.9)) if moved.any() else 0.0
    op_min, scale_min = math.log(0.005 / 0.995), math.log(0.01)
    cap = 2 * n
    outs = [(torch.empty((cap, 4), device=dev), torch.empty(cap, device=dev), torch.empty((cap, C), device=dev))
            for _ in range(3)]
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    work = torch.empty(igs.densify_work_bytes(n), dtype=torch.uint8, device=dev)
    args = (ts.scene, ts.m_views, ts.v_views, 3, 1, ts.accum, ts.vis, op_min, tau_g, scale_min, outs[0], outs[1],
            outs[2], count, work)
    igs.densify(*args)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        igs.densify(*args, stream=stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / reps
    k = int(count.item())
    op = ts.op.cpu().numpy()
    kept = int((~(op < op_min)).sum())
    divided = (k - kept) // 7
    row = 4 * (5 + C)
    nbytes = 2 * 28 * n + 2 * 3 * row * (kept - divided) + divided * (row + 8 * 3 * row)
    gbs = nbytes / (ms / 1e3) / 1e9
    ts.accum = ts.vis = None
    return {"n": n, "steps_tracked": steps, "step_ms": round(plain_ms, 4), "step_ms_with_statistic":
            round(tracked_ms, 4), "tau_g": tau_g, "with_gradient": int(moved.sum()), "kept": kept, "deleted": n - kept, "divided": divided,
            "out": k, "densify_ms": round(ms, 4),
            "roofline": {"bound": "hbm", "bytes": nbytes, "achieved": round(gbs, 1), "peak": peak_hbm,
                         "unit": "GB/s", "frac": round(gbs / peak_hbm, 4)}}


def run_merge3d(ts, stream, dev, peak_hbm, reps=3, cells=128):
    """Merging of the training scene's Gaussians (igs_merge) into new buffers: a
    grid of `cells` cells per axis over the scene's bounding box, the Gaussians
    with sigma at most the median eligible. Groups are counted on the host from
    the same FP32 cell rule. Bandwidth over the pass's algorithmic bytes: 20 B per
    Gaussian (mean, scale and opacity for its cell key), 2 x 3 rows per kept
    Gaussian (parameters and moments read and written), one row read per member
    of a merged cell and 3 rows written per merged Gaussian (row = 4 (5 + C) B)."""
    import numpy as np
    import torch

    from paper_2403_14244_gb300 import igs

    n, C = ts.n, ts.C
    ms = ts.ms.cpu().numpy()
    op = ts.op.cpu().numpy()
    lo = ms[:, :3].min(0)
    h = float((ms[:, :3].max(0) - lo).max()) / cells * 1.0001
    smax = float(np.median(ms[:, 3]))
    inv = np.float32(1.0) / np.float32(h)
    cell = np.floor((ms[:, :3] - lo.astype(np.float32)) * inv)
    with np.errstate(invalid="ignore", over="ignore"):
        ok = (np.isfinite(ms[:, :3]).all(1) & (ms[:, 3] <= np.float32(smax)) & (1 / (1 + np.exp(-op.astype(np.float64))) > 0)
              & (cell >= 0).all(1) & (cell < 1024).all(1))
    ci = cell[ok].astype(np.int64)
    _, cnt = np.unique(ci[:, 0] | (ci[:, 1] << 10) | (ci[:, 2] << 20), return_counts=True)
    groups, members = int((cnt >= 2).sum()), int(cnt[cnt >= 2].sum())
    outs = [(torch.empty((n, 4), device=dev), torch.empty(n, device=dev), torch.empty((n, C), device=dev))
            for _ in range(3)]
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    work = torch.empty(igs.merge_work_bytes(n), dtype=torch.uint8, device=dev)
    args = (ts.scene, ts.m_views, ts.v_views, 3, 1, [float(x) for x in lo], h, smax, outs[0], outs[1], outs[2], count,
            work)
    igs.merge(*args)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        igs.merge(*args, stream=stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms_t = a.elapsed_time(b) / reps
    k = int(count.item())
    kept = n - members
    row = 4 * (5 + C)
    nbytes = 20 * n + 2 * 3 * row * kept + row * members + 3 * row * groups
    gbs = nbytes / (ms_t / 1e3) / 1e9
    return {"n": n, "cells_per_axis": cells, "cell": h, "scale_max_log": smax, "merged_cells": groups,
            "members": members, "out": k, "out_expected": kept + groups, "merge_ms": round(ms_t, 4),
            "roofline": {"bound": "hbm", "bytes": nbytes, "achieved": round(gbs, 1), "peak": peak_hbm,
                         "unit": "GB/s", "frac": round(gbs / peak_hbm, 4)}}


def run_ssim_steps(ts, cam_s, targets, stream, dev, steps, peak_hbm, lam=0.2):
    """The same training step with the paper's loss (1 - lam) L1 + lam (1 - SSIM)
    in place of L1: steps/s, stage times, and the loss kernels' bandwidth over
    their algorithmic bytes (per image entry: img, target read and three partial
    maps written by the forward kernel; the maps, img and target read and the
    gradient written by the backward kernel: 44 bytes)."""
    import torch

    stages = ("project", "bin_sort", "blend_fwd", "l1_ssim", "blend_bwd", "project_bwd_adam_next")
    V = len(cam_s)
    ts.ssim_lambda = lam
    try:  # as the headline step: each step projects the next view in its last pass
        for k in range(3):
            ts.step(cam_s[k % V], targets[k % V], next_cam=cam_s[(k + 1) % V])
        torch.cuda.synchronize(dev)
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stage_ev = []
        start.record(stream)
        for k in range(3, 3 + steps):
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)]
            evs[0].record(stream)
            it = iter(evs[1:])
            ts.step(cam_s[k % V], targets[k % V], marks=lambda name, it=it: next(it).record(stream),
                    next_cam=cam_s[(k + 1) % V])
            stage_ev.append(evs)
        end.record(stream)
        torch.cuda.synchronize(dev)
    finally:
        ts.ssim_lambda = 0.0
    ms = start.elapsed_time(end) / steps
    stage_ms = {s: sum(e[i].elapsed_time(e[i + 1]) for e in stage_ev) / steps for i, s in enumerate(stages)}
    stage_ms.pop("project")  # (inside the previous step's last pass)
    entries = targets[0].numel()
    nbytes = 44 * entries
    gbs = nbytes / (stage_ms["l1_ssim"] / 1e3) / 1e9
    return {"lambda": lam, "steps": steps, "steps_per_s": round(1e3 / ms, 3), "ms_per_step": round(ms, 4),
            "stage_ms": {s: round(v, 4) for s, v in stage_ms.items()},
            "l1_ssim_roofline": {"bound": "hbm", "bytes": nbytes, "achieved": round(gbs, 1), "peak": peak_hbm,
                                 "unit": "GB/s", "frac": round(gbs / peak_hbm, 4)}}


def run_extra(dev, np, tile=32):
    """1080p forward frames/s and fwd+bwd steps/s on the 1M clustered SH3 scene."""
    import torch

    from paper_2403_14244_gb300 import igs, scenes
    from paper_2403_14244_gb300.render import Renderer

    sc, cam, target = scenes.workload_fwd_bwd_1m()
    scene = igs.Scene.from_numpy(sc, dev)
    r = Renderer(tile=tile, sh_degree=3, param_mode=0, device=dev)
    c = igs.camera(cam)
    img, f = r.run_forward(scene, c, check=True)
    tg = torch.from_numpy(target).to(dev)
    loss = torch.zeros(1, device=dev)
    dimg = torch.empty_like(img)
    g2d = torch.empty((scene.n, 8), device=dev)
    grads = (torch.empty_like(scene.means_sigma), torch.empty_like(scene.opacity), torch.empty_like(scene.color))
    reps = 50

    def fwd():
        igs.project(scene, c, r.opts, f)
        igs.bin_sort(f, r.opts)
        igs.render_fwd(f, r.opts, img)

    def fwdbwd():
        fwd()
        igs.l1_loss(img, tg, loss, dimg)
        igs.render_bwd(scene, c, r.opts, f, dimg, g2d, *grads)

    out = {"fwd_256_4k": run_small_forward(dev)}
    for name, fn in (("fwd_1080p_1M", fwd), ("fwd_bwd_1080p_1M", fwdbwd)):
        for _ in range(5):
            fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / reps
        out[name] = {"ms": round(ms, 4), "per_s": round(1e3 / ms, 1)}
    st, info = igs.frame_status(f)
    assert st == igs.OK
    out["fwd_bwd_1080p_1M"]["entries_M"] = info[0]
    del scene, r, f, img, g2d, grads
    torch.cuda.empty_cache()
    out["octree_init"] = run_octree(dev)
    out["fit2d_512"] = run_fit2d(dev)
    out["batched_32view_2M"] = run_batched(dev)
    out["serve_4scenes_poisson"] = run_serving(dev)
    return out


def run_small_forward(dev, reps=200):
    """The 4,096-Gaussian forward at 256x256 with 16-pixel tiles (project, bin and
    sort, blend): microseconds per frame, launch-bound at this size (no
    roofline claim), eager launches and one CUDA graph of the three calls."""
    import torch

    from paper_2403_14244_gb300 import igs, scenes
    from paper_2403_14244_gb300.render import Renderer

    sc, cam = scenes.workload_forward_4k()
    scene = igs.Scene.from_numpy(sc, dev)
    r = Renderer(tile=16, device=dev)
    c = igs.camera(cam)
    img, f = r.run_forward(scene, c, check=True)

    def fwd(stream=None):
        igs.project(scene, c, r.opts, f, stream)
        igs.bin_sort(f, r.opts, stream)
        igs.render_fwd(f, r.opts, img, stream)

    out = {"n": 4096, "image": [256, 256], "tile": 16}
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(10):
        fwd()
    torch.cuda.synchronize(dev)
    a.record()
    for _ in range(reps):
        fwd()
    b.record()
    torch.cuda.synchronize(dev)
    out["eager_us_per_frame"] = round(1e3 * a.elapsed_time(b) / reps, 2)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            fwd(s)
    torch.cuda.current_stream(dev).wait_stream(s)
    for _ in range(10):
        g.replay()
    torch.cuda.synchronize(dev)
    a.record()
    for _ in range(reps):
        g.replay()
    b.record()
    torch.cuda.synchronize(dev)
    out["graph_us_per_frame"] = round(1e3 * a.elapsed_time(b) / reps, 2)
    out["frames_per_s"] = round(1e6 / out["graph_us_per_frame"], 1)
    st, info = igs.frame_status(f)
    assert st == igs.OK
    out["entries"] = info[0]
    return out


def cpu_configs(budget_s=20.0):
    """The CPU oracle on the two smaller workloads, beside the GPU numbers in
    `extra` (a baseline, not a target): the 4,096-Gaussian 256x256 forward
    (repeated for about a second), and one full forward and one full forward +
    adjoint of the 1M-Gaussian SH3 1080p scene (the adjoint includes its own
    forward; skipped when the forward alone used more than half the budget)."""
    import oracle
    from paper_2403_14244_gb300 import scenes

    oracle.build()
    out = {"cores": oracle.num_threads(), "kind": "oracle", "cpu": _cpu_model()}
    sc, cam = scenes.workload_forward_4k()
    t0 = time.perf_counter()
    reps = 0
    while time.perf_counter() - t0 < 1.0 or reps < 3:
        oracle.render(sc, cam, mode=1)
        reps += 1
    out["fwd_256_4k"] = {"ms_per_frame": round(1e3 * (time.perf_counter() - t0) / reps, 3), "frames": reps}
    sc, cam, target = scenes.workload_fwd_bwd_1m()
    t0 = time.perf_counter()
    ref = oracle.render(sc, cam, mode=1)
    t_fwd = time.perf_counter() - t0
    row = {"fwd_ms": round(1e3 * t_fwd, 1)}
    if t_fwd < budget_s / 2:
        _, G = oracle.l1(ref["img"], target)
        t0 = time.perf_counter()
        oracle.backward(sc, cam, G, mode=1)
        row["fwd_bwd_ms"] = round(1e3 * (time.perf_counter() - t0), 1)
    out["fwd_bwd_1080p_1M"] = row
    return out


def run_octree(dev, n=2_000_000, levels=7, k_max=500_000, reps=3):
    """Octree initialisation of 3D Gaussians from a seeded coloured point set
    (n points: 64 clusters and a uniform background in [-1, 1]^3, colours with
    structure at several scales), cells down to side 2 / 2^levels, at most
    k_max Gaussians: time per call (statistics, up-sweep, radix selection of
    the splits, emission) and the Gaussians made."""
    import torch

    from paper_2403_14244_gb300 import igs, scenes

    p, c = scenes.point_cloud(n, seed=8)
    tp, tc = torch.from_numpy(p).to(dev), torch.from_numpy(c).to(dev)
    igs.octree_init(tp, tc, (-1, -1, -1), 2.0, levels, k_max)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(reps):
        ms, _, _ = igs.octree_init(tp, tc, (-1, -1, -1), 2.0, levels, k_max)
    torch.cuda.synchronize(dev)
    ms_per = (time.perf_counter() - t0) / reps * 1e3
    return {"points": n, "levels": levels, "k_max": k_max, "gaussians": int(ms.shape[0]),
            "ms_per_call": round(ms_per, 3), "note": "includes the count read-back (one synchronisation)"}


def run_fit2d(dev, iters=2000, side=512, min_cell=3):
    """The paper's 2D experiment at its Table 2 settings (support D in {15, 50}
    pixels, K in {1000, 2000} particles): QuadTree initialisation, then `iters`
    iterations of render + (0.8 L1 + 0.2 (1 - SSIM)) + adjoint + Adam, replayed
    from a CUDA graph of 50 iterations, on a seeded synthetic 512x512 image.
    Reports the time of the initialisation and of the iterations, the per-kernel
    split of one eager iteration, and the fit (loss, PSNR) before and after."""
    import math

    import torch

    from paper_2403_14244_gb300 import scenes
    from paper_2403_14244_gb300.fit2d import Fit2D

    target = torch.from_numpy(scenes.fit2d_image(side, 6)).to(dev)
    paper_min = {(15, 1000): 0.12, (50, 1000): 0.13, (15, 2000): 0.25, (50, 2000): 0.27}
    out = {"image": [side, side], "iters": iters, "min_cell": min_cell, "lambda": 0.2,
           "paper_table2_iso_minutes": "context only (2D image and hardware not given)"}

    def psnr(f):
        f.render()
        mse = float(((f.img - f.target) ** 2).mean())
        return round(10 * math.log10(1.0 / mse), 2)

    Fit2D(target, 16, 15.0, min_cell=min_cell)   # loads the kernels: the timed set-ups below exclude that

    for (D, K), ref_min in paper_min.items():
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record()
        f = Fit2D(target, K, float(D), min_cell=min_cell)
        b.record()
        torch.cuda.synchronize(dev)
        init_ms = a.elapsed_time(b)
        psnr0 = psnr(f)
        # per-kernel split of one eager iteration
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record()
        from paper_2403_14244_gb300 import igs
        igs.fit2d_render(f.particles, f.D, f.img)
        ev[1].record()
        igs.l1_ssim_loss(f.img, f.target, f.lam, f.loss, f.dimg, f.work, ssim=f.ssim)
        ev[2].record()
        igs.fit2d_backward(f.particles, f.D, f.dimg, f.grad)
        ev[3].record()
        igs.fit2d_adam(f.particles, f.grad, f.m, f.v, f.lr, f.state)
        ev[4].record()
        torch.cuda.synchronize(dev)
        loss0 = float(f.loss)
        split = {n: round(ev[i].elapsed_time(ev[i + 1]), 4)
                 for i, n in enumerate(("render", "loss", "backward", "adam"))}
        f.capture(inner=50)
        torch.cuda.synchronize(dev)
        a.record()
        n = f.run(iters)
        b.record()
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b)
        f.render()
        igs.l1_ssim_loss(f.img, f.target, f.lam, f.loss, f.dimg, f.work, ssim=f.ssim)
        out[f"D{D}_K{K}"] = {
            "particles": f.k, "init_ms": round(init_ms, 3), "iter_ms": round(ms / n, 4),
            "iters_per_s": round(1e3 * n / ms, 1),
            "fit_minutes": round((init_ms + ms) / 60000.0, 6), "paper_iso_minutes": ref_min,
            "eager_split_ms": split, "loss_first": round(loss0, 5), "loss_last": round(float(f.loss), 5),
            "ssim_last": round(float(f.ssim), 4), "psnr_init_db": psnr0, "psnr_last_db": psnr(f)}
        del f
    out["densify_D15"] = run_fit2d_densify(dev, target, iters, min_cell, psnr)
    return out


def run_fit2d_densify(dev, target, iters, min_cell, psnr, D=15.0, k0=256, capacity=1000, every=500):
    """Densify / prune during the 2D fit: start from a QuadTree of k0 particles;
    every `every` iterations delete particles with max |A| < 0.01 and divide
    those whose mean position-gradient norm is in the top quarter (threshold
    read from the accumulated statistic on the host) into four half-scale
    children, within `capacity` particles. Reports the densify kernel's time,
    the particle counts and the fit, to compare with the QuadTree started at
    `capacity` particles above."""
    import numpy as np
    import torch

    from paper_2403_14244_gb300.fit2d import Fit2D

    f = Fit2D(target, k0, D, min_cell=min_cell)
    f.track_grad_norm()
    f.capture(inner=50)
    counts, dens_ms = [f.k], []
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    done = 1
    while done < iters:
        done += f.run(min(every, iters - done))
        if done >= iters:
            break
        tau_g = float(np.quantile(f.accum.cpu().numpy(), 0.75)) / f.accum_iters
        a.record()
        f.densify(0.01, tau_g, 0.0, capacity)   # includes the count read-back
        b.record()
        torch.cuda.synchronize(dev)
        dens_ms.append(round(a.elapsed_time(b), 4))
        counts.append(f.k)
        f.capture(inner=50)
        done += 1
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    return {"D": D, "k_start": k0, "capacity": capacity, "every": every, "iters": done, "particles": counts,
            "densify_ms": dens_ms, "wall_s": round(wall, 3), "psnr_last_db": psnr(f)}


def run_batched_fixed(dev, n, views, warm, reps):
    """One batched render of `views` sphere poses of an n-Gaussian RGB scene at
    tile 32 / staging 64, captured once and replayed: ms per render (for a
    launch list or a counter capture of the batched path without the tuner)."""
    import torch

    from paper_2403_14244_gb300 import igs, scenes
    from paper_2403_14244_gb300.batch import BatchRenderer

    scene = igs.Scene.from_numpy(scenes.uniform_scene(n, 4), dev)
    cams = [igs.camera(c) for c in scenes.sphere_cameras(views, 4)]
    br = BatchRenderer(scene, cams, tile=32, blend_batch=64, device=dev)
    br.capture()
    for _ in range(warm):
        br.replay()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        br.replay()
    b.record()
    torch.cuda.synchronize(dev)
    br.check()
    ms = a.elapsed_time(b) / max(reps, 1)
    return {"n": n, "views": views, "tile": 32, "blend_batch": 64, "groups": [len(g) for g in br.groups],
            "entries": int(sum(br.entries)), "replays": reps, "ms": round(ms, 3)}


def run_batched(dev, reps=10):
    """32 views (sphere poses, mixed 360p..1440p) of a 2M-Gaussian RGB scene:
    autotuned batched graph replays vs a loop of one-view renders, frames/s."""
    import torch

    from paper_2403_14244_gb300 import igs, scenes
    from paper_2403_14244_gb300.batch import BatchRenderer, autotune
    from paper_2403_14244_gb300.render import Renderer

    sc = scenes.uniform_scene(2_000_000, 4)
    scene = igs.Scene.from_numpy(sc, dev)
    cams = [igs.camera(c) for c in scenes.sphere_cameras(32, 4)]
    cache = os.environ.get("IGS_AUTOTUNE_CACHE")  # where to keep the tuner's choice, if anywhere
    (tile, bb), timings = autotune(scene, cams, candidates=[(8, 64), (16, 64), (16, 256), (32, 64), (32, 512)], reps=3,
                                   cache_path=cache, use_cache=False, device=dev)
    br = BatchRenderer(scene, cams, tile=tile, blend_batch=bb, device=dev)
    br.capture()
    for _ in range(2):
        br.replay()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        br.replay()
    b.record()
    torch.cuda.synchronize(dev)
    br.check()
    batched_ms = a.elapsed_time(b) / reps
    entries = sum(br.entries)
    del br
    torch.cuda.empty_cache()
    # one view at a time through the one-view path (capacity from a checked first
    # pass), at each tile size; the best one is the baseline
    loop = {}
    for lt in (16, 32):
        r = Renderer(tile=lt, device=dev)
        imgs = {}
        for c in cams:
            imgs[(c.width, c.height)] = r.run_forward(scene, c, check=True)[0]
        for _ in range(2):
            for c in cams:
                r.run_forward(scene, c, img=imgs[(c.width, c.height)], check=False)
        torch.cuda.synchronize(dev)
        a.record()
        for _ in range(reps):
            for c in cams:
                r.run_forward(scene, c, img=imgs[(c.width, c.height)], check=False)
        b.record()
        torch.cuda.synchronize(dev)
        loop[lt] = a.elapsed_time(b) / reps
        del r, imgs
        torch.cuda.empty_cache()
    lt = min(loop, key=loop.get)
    return {"views": len(cams), "tile": tile, "blend_batch": bb, "entries": entries,
            "autotune_ms": {k: round(v, 3) for k, v in timings.items()},
            "batched_ms": round(batched_ms, 3), "batched_frames_per_s": round(len(cams) * 1e3 / batched_ms, 1),
            "loop_ms_by_tile": {str(k): round(v, 3) for k, v in loop.items()}, "loop_tile": lt,
            "loop_frames_per_s": round(len(cams) * 1e3 / loop[lt], 1)}


SERVE_RATES = (200.0, 800.0, 1100.0, 1500.0)
SERVE_MODES = {"slots1": (1, 1), "slots4": (4, 1), "slots4_group8": (4, 8)}


def run_serving(dev, n_req=2000, warm=200, rate=200.0, budget=8 << 30, seed=5, tile=32):
    """Four resident scenes (0.5, 1, 2, 4M Gaussians), open-loop Poisson arrivals,
    random scene, sphere pose, 480p..2160p, on the same arrival pattern (gaps
    scaled) at each rate of SERVE_RATES (the workload's own 200/s first) and all
    at once (burst); served strictly one at a time (slots1), with 4 slots
    (continuous batching), and with 4 slots whose queued requests of one scene
    share a batched chain (up to 8 views)."""
    import threading

    import numpy as np
    import torch

    from paper_2403_14244_gb300 import igs, scenes

    rng = np.random.default_rng(seed)
    scs = [igs.Scene.from_numpy(scenes.uniform_scene(int(m * 1_000_000), 50 + k), dev)
           for k, m in enumerate((0.5, 1, 2, 4))]
    total = n_req + warm
    gaps = rng.exponential(1.0 / rate, size=total)
    which = rng.integers(0, 4, size=total)
    cams = scenes.sphere_cameras(total, seed, resolutions=scenes.RESOLUTIONS_SERVE)
    ring = 48
    bufs = {(w, h): [torch.empty((3, h, w), device=dev) for _ in range(ring)] for w, h in scenes.RESOLUTIONS_SERVE}
    out = {}

    def serve(slots, gaps, group=1):
        srv = igs.Server(pool_bytes=budget, slots=slots, tile=tile, device=dev, group=group)
        sids = [srv.add_scene(sc) for sc in scs]
        cam_s = [igs.camera(c) for c in cams]
        ids = [None] * total
        done = [threading.Event() for _ in range(total)]
        timings = [None] * total
        use = {k: [None] * ring for k in bufs}  # request last using each buffer

        def poller():
            for i in range(total):
                while ids[i] is None:
                    time.sleep(1e-4)
                st, t = srv.poll(ids[i], timeout_s=120.0)
                timings[i] = (st, t)
                done[i].set()

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        arrive = time.perf_counter()
        for i in range(total):
            arrive += gaps[i]
            c = cam_s[i]
            key = (c.width, c.height)
            slot = i % ring
            prev = use[key][slot]
            if prev is not None:
                done[prev].wait()
            use[key][slot] = i
            delay = arrive - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids[i] = srv.submit(sids[which[i]], c, bufs[key][slot])
        th.join()
        stats = srv.stats()
        srv.close()
        meas = [timings[i][1] for i in range(warm, total)]
        bad = sum(1 for i in range(warm, total) if timings[i][0] != igs.OK)
        lat = np.array([(t["done_ns"] - t["arrival_ns"]) / 1e6 for t in meas])
        span = (max(t["done_ns"] for t in meas) - min(t["arrival_ns"] for t in meas)) / 1e9
        grp = [t["group"] for t in meas]
        return {"p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "max_ms": round(float(lat.max()), 3), "frames_per_s": round((n_req - bad) / span, 1), "failed": bad,
                "pool_peak_bytes": int(stats["pool_peak"]), "retries": int(sum(t["retries"] for t in meas)),
                "mean_group": round(float(np.mean(grp)), 2)}

    for r in SERVE_RATES:
        for name, (slots, group) in SERVE_MODES.items():
            if r == rate and name == "slots4_group8":
                continue  # at the workload's own rate requests rarely wait: grouping has nothing to group
            out[f"poisson{int(r)}_{name}"] = serve(slots, gaps * (rate / r), group)
    # the same requests submitted back to back: the throughput each mode can sustain
    for name, (slots, group) in SERVE_MODES.items():
        out[f"burst_{name}"] = serve(slots, np.zeros(total), group)
    out["tile"] = tile
    out["requests"] = n_req
    out["warmup"] = warm
    out["rate_per_s"] = rate
    out["pool_bytes"] = budget
    return out


# ------------------------------------------------------------ CPU oracle ----

def oracle_step(sc, cam, target, lam=0.0):
    """One training step of the CPU oracle: FP64 forward + adjoint (row-list
    mode, all host cores), L1 loss (or (1 - lam) L1 + lam (1 - SSIM)), Adam over
    all parameters."""
    import numpy as np

    import oracle

    fwd = oracle.render(sc, cam, mode=1)
    if lam > 0:
        loss, _, G = oracle.l1_ssim(fwd["img"], target, lam=lam)
    else:
        loss, G = oracle.l1(fwd["img"], target)
    g = oracle.backward(sc, cam, G, mode=1)
    flat_g = np.concatenate([np.concatenate([g["d_means"], g["d_sigma"][:, None]], 1).reshape(-1), g["d_opac"],
                             g["d_color"].reshape(-1)])
    p = np.concatenate([sc.means_sigma.reshape(-1), sc.opacity, sc.color.reshape(-1)]).astype(np.float64)
    oracle.adam(p, flat_g, np.zeros(p.size), np.zeros(p.size), lr=1e-3, t=1)
    return loss


def cpu_baseline(sc, cams, budget_s, lam=0.0):
    import oracle
    from paper_2403_14244_gb300 import scenes

    oracle.build()
    t0 = time.perf_counter()
    steps = 0
    while True:
        oracle_step(sc, cams[steps % len(cams)], scenes.train_target(steps % len(cams)), lam=lam)
        steps += 1
        if time.perf_counter() - t0 >= budget_s or steps >= 8:
            break
    dt = time.perf_counter() - t0
    return {"value": round(steps / dt, 5), "unit": "steps/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{steps} full training step(s) of the same workload (views 0..{steps - 1}): FP64 forward + "
                      f"adjoint over all 1297x840 pixels, {'L1' if lam == 0 else 'L1 + SSIM'}, Adam over all "
                      f"53 x 3M parameters; {dt:.1f} s",
            "cpu": _cpu_model()}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


REF_BUDGET_S = 240.0


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle on the same workload and metric, in
    whole training steps (FP64 forward + adjoint over every pixel of one view,
    L1, Adam over all 53 n parameters), the views cycling as in the GPU arm. One
    untimed warm-up step (the oracle has no state to warm beyond its first
    call), then up to --steps timed steps; the timed region stops once it has
    used REF_BUDGET_S seconds, and `steps` then reports the steps it timed."""
    if rank != 0:
        return
    import oracle
    from paper_2403_14244_gb300 import scenes

    oracle.build()
    sc, cams = scenes.workload_train_3m(n=args.n)
    V = len(cams)
    warm = min(args.warmup, 1)
    for k in range(warm):
        oracle_step(sc, cams[k % V], scenes.train_target(k % V), lam=args.ssim)
    t0 = time.perf_counter()
    done = 0
    while done < args.steps:
        oracle_step(sc, cams[done % V], scenes.train_target(done % V), lam=args.ssim)
        done += 1
        if time.perf_counter() - t0 >= REF_BUDGET_S:
            break
    dt = time.perf_counter() - t0
    value = done / dt
    sample = (f"{done} whole training steps (views 0..{min(done, V) - 1}, cycling): oracle FP64 forward + adjoint "
              f"over all 1297x840 pixels, {'L1' if args.ssim == 0 else 'L1 + SSIM'}, Adam over all 53 x {args.n} "
              f"parameters; {warm} untimed warm-up step; {dt:.1f} s timed")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "steps/s", "n_gpus": world,
        "steps": done, "steps_requested": args.steps, "warmup": warm, "warmup_requested": args.warmup,
        "ms_per_step": round(1e3 * dt / done, 2), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded generators, no dataset)",
        "config": workload_config(args, args.n, world),
        "cpu_baseline": {"value": round(value, 6), "unit": "steps/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample, "cpu": _cpu_model()},
        "e2e": {"value": round(value, 6), "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.only == "merge":
        import torch
        dev = torch.device("cuda", local)
        torch.cuda.set_device(dev)
        _, _, _, ts, _, _, _ = build_workload(args.n, dev, args.footprint, args.tile)
        print(json.dumps({"merge_3M": run_merge3d(ts, torch.cuda.current_stream(dev), dev, load_peaks()[0])}))
        return
    if args.only == "batched":
        import torch
        dev = torch.device("cuda", local)
        torch.cuda.set_device(dev)
        print(json.dumps({"batched": run_batched_fixed(dev, args.batch_n, args.batch_views, args.warmup, args.steps)}))
        return
    run_mine(args, world, rank, local)


if __name__ == "__main__":
    main()
