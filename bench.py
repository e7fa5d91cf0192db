#!/usr/bin/env python3
"""Benchmark of the GB300 Gaussian rasterizer + pose gradient.

Workload (synthetic, seeded): 1,000,000 Gaussians over a 1 km x 1 km aerial
scene (SH degree 3), one 1920x1080 view (f = 1400) from 300 m pitched 30 deg.
A step is one pose-refinement iteration of the whole hot path: projection,
tile binning + depth sort, front-to-back compositing of RGB/depth/alpha, the
L1 photometric + 0.1 L1 depth loss and its se(3) pose gradient (fp64
reduction). ``value`` is rendered-and-differentiated Mpix/s (whole job); the
line also reports forward-only Mpix/s, pose-gradient iterations/s and the
batched-vs-single-pose factor on the mixed-resolution batch (84 candidate
poses, 2M Gaussians with 32 BF16 feature channels).

L2 is flushed (256 MB write) between timed steps, outside the timed events.
``python bench.py [--gpus N --steps K --warmup W] [--impl reference]``; for
N > 1 run under torchrun (one rank per GPU, independent poses per rank).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpix/s fwd and pose-grad iters/s, 1M Gaussians @1080p; batched vs single-pose"
WORKLOAD = ("aerial 1M Gaussians SH3, 1920x1080 f=1400, pose-gradient step (fwd + L1 rgb/depth loss + se(3) "
            "gradient)")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20
# fp32 operations of one (pixel, Gaussian) evaluation on the skip path:
# dx, dy, dx^2, dy^2, A dx^2, C dy^2 (+), x(-1/2), dx dy, B dx dy (+), o e^p, min, 2 compares
FLOPS_PER_EVAL = 14
# additional fp32 operations of a blended evaluation in the tangent pass (FMA = 2):
# blend 12 (1 - a, T', w = a T, C, D += w (c, z)); tangent 168: -dpower/dxi over 6
# directions (5 FMA each) 60, dalpha 6, dw = dalpha T + a dT 18, dT 6, dC 36,
# colour rows (3 x 3 FMA) 18, dD 24
FLOPS_PER_BLEND = 180
# DRAM bytes (read + write) of one tangent-pass launch on this workload, from
# one ncu capture of this kernel (dram__bytes_read.sum + dram__bytes_write.sum);
# None whenever the kernel has changed since that capture
COMPOSITE_DRAM_BYTES = 82_540_288  # 79,541,760 read + 2,998,528 written (the tuned 128 / 3 variant)
# Visibility reverse pass (Algorithm 1): a (pixel, Gaussian) evaluation shares
# the forward's FLOPS_PER_EVAL; a blended pair adds the transmittance
# division, weight, colour sum and running sum (8), dL/dpower and the five
# monomials (7) and their share of the per-record sums over pixels (6).
FLOPS_PER_VIS_BLEND = 21
# DRAM bytes of one reverse-pass launch (ncu, same kernel): 37,543,680 read + 72,448 written
VIS_BACKWARD_DRAM_BYTES = 37_616_128
# PnP scoring (Eq. 10 RANSAC): one (solution, match) pair is p = R X + t (9 FMA),
# x - a z, y - b z (2 FMA), the scaled squares (2 mul + 1 FMA), tau z twice (2 mul),
# the threshold difference (1 FMA) and 2 compares: 33 fp32 operations (FMA = 2)
FLOPS_PER_PNP_PAIR = 33
# DRAM bytes of one scoring launch on this workload (ncu, 313 solutions x 491,752 matches)
PNP_SCORE_DRAM_BYTES = 11_834_880


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gsr", choices=["gsr", "reference"])
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-refine", action="store_true")
    p.add_argument("--no-large", action="store_true")
    p.add_argument("--no-pmm", action="store_true")
    p.add_argument("--no-vis", action="store_true")
    p.add_argument("--no-dense", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-errors", action="store_true")
    p.add_argument("--only", default="", choices=["", "batched"],
                   help="run one section alone (for profiling) and print its result")
    p.add_argument("--batched-views", type=int, default=0, help="the batched section on its first N views only")
    p.add_argument("--pin", default="", help="launch configurations to use instead of the autotuner's for the "
                   "headline view, e.g. 'pose_grad=2,0,8;forward=2,0,8' (variant, CTAs per SM, grid multiple)")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# Replicas only: each rank renders its own query pose of the same scene (independent
# units, no collective on the data path); timing takes the slowest rank, and the
# whole-job value counts every rank's pixels.
def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mpix_per_s(world: int, pixels: int, ms: float) -> float:
    """Whole-job throughput: every rank's pixels over the slowest rank's step time."""
    return world * pixels / (ms * 1e-3) / 1e6


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="gsr_clocks_", suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.bus_id:
            cmd[1:1] = ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        loaded = [r for r in rows if len(r) > 9 and (num(r[9]) or 0) >= 50] or rows
        sm = [num(r[1]) for r in loaded if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(loaded),
                "power_w_max": max(pw) if pw else None,
                "window": "all GPU measurement sections of this run (utilization >= 50 % for the median)"}


def peaks():
    try:
        return json.load(open(PEAKS_FILE)), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------------------- workload
def make_workload(rank: int):
    from paper_2507_15683_gb300 import synth
    scene = synth.aerial_scene(2, 1_000_000)
    cam = synth.aerial_camera()
    T_ref = synth.aerial_pose()
    T_q = synth.perturb_pose(T_ref, synth.rng(100 + rank), 2.0, 5.0)
    return scene, cam, T_ref, T_q


def cpu_baseline(scene, cam, T_ref, T_q, budget_s: float):
    """The fp64 oracle as it stands, on a bounded pixel sample of the same frame."""
    from oracle import oracle as O
    O.build()
    n_thr = os.cpu_count() or 1
    H, W = cam["height"], cam["width"]
    t0 = time.perf_counter()
    ref = O.render(scene, cam, T_ref, geom64=True, n_threads=n_thr)  # target frame (not timed below)
    t_ref = time.perf_counter() - t0
    trgb = ref["rgb"].T.reshape(3, H, W).astype(np.float32)
    tdep = ref["depth"].reshape(H, W).astype(np.float32)
    g = np.random.default_rng(0)
    n_pix = 16384
    while True:
        pix = np.sort(g.choice(H * W, n_pix, replace=False))
        w = np.zeros((H, W), np.float32)
        w.reshape(-1)[pix] = 1.0
        t0 = time.perf_counter()
        r = O.render(scene, cam, T_q, geom64=True, want_grad=True, pixels=pix, target_rgb=trgb, target_depth=tdep,
                     pixel_weight=w, n_threads=n_thr)
        dt = time.perf_counter() - t0
        if dt > budget_s / 3 or n_pix >= H * W:
            break
        n_pix = min(H * W, int(n_pix * max(2.0, budget_s / 2 / max(dt, 1e-3))))
    # the same step on one core, on a sample sized for about a fifth of the budget
    n1 = max(1024, min(H * W, int(n_pix * (budget_s / 5) / max(dt * n_thr, 1e-3))))
    pix1 = np.sort(g.choice(H * W, n1, replace=False))
    w1 = np.zeros((H, W), np.float32)
    w1.reshape(-1)[pix1] = 1.0
    t0 = time.perf_counter()
    O.render(scene, cam, T_q, geom64=True, want_grad=True, pixels=pix1, target_rgb=trgb, target_depth=tdep,
             pixel_weight=w1, n_threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": n_pix / dt / 1e6, "unit": "Mpix/s", "cores": n_thr, "kind": "oracle",
            "sample": "fp64 oracle pose-gradient step (projection of all 1M Gaussians, binning, fp64 "
                      "compositing + forward-mode se(3) gradient) on %d random pixels of the 1080p frame; "
                      "%.2f s per step" % (n_pix, dt),
            "single_thread": {"value": n1 / dt1 / 1e6, "unit": "Mpix/s", "cores": 1,
                              "sample": "the same step on %d random pixels, %.2f s" % (n1, dt1)},
            "cpu_model": cpu_model(),
            "loss": r["loss"], "target_render_s": t_ref}


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def run_reference(args):
    """Reference arm: the CPU oracle, timed on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    scene, cam, T_ref, T_q = make_workload(0)
    from oracle import oracle as O
    O.build()
    n_thr = os.cpu_count() or 1
    H, W = cam["height"], cam["width"]
    ref = O.render(scene, cam, T_ref, geom64=True, n_threads=n_thr)
    trgb = ref["rgb"].T.reshape(3, H, W).astype(np.float32)
    tdep = ref["depth"].reshape(H, W).astype(np.float32)
    n_pix = H * W  # the whole frame per step, as the GPU arm (about 0.75 s on 16 cores)

    def step():
        O.render(scene, cam, T_q, geom64=True, want_grad=True, target_rgb=trgb, target_depth=tdep,
                 n_threads=n_thr)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    v = n_pix / dt / 1e6
    line = {"metric": METRIC, "value": v, "unit": "Mpix/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "gaussians": 1_000_000, "width": W, "height": H, "sh_degree": 3,
                       "sample_pixels": n_pix},
            "cpu_baseline": {"value": v, "unit": "Mpix/s", "cores": n_thr, "kind": "oracle",
                             "sample": "fp64 oracle pose-gradient step (projection of all 1M Gaussians, binning, "
                                       "fp64 compositing + forward-mode se(3) gradient) on the whole %dx%d frame "
                                       "per step" % (W, H)},
            "e2e": {"value": v, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    if args.only == "batched":  # one section alone, for profiling
        torch.cuda.set_device(0)
        from paper_2507_15683_gb300 import gsr, synth
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        print(json.dumps(bench_batched(gsr, synth, torch, flush, max(1, args.steps), args.warmup,
                                       args.batched_views or None)), flush=True)
        return
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2507_15683_gb300 import gsr, synth

    scene, cam, T_ref, T_q = make_workload(rank)
    H, W = cam["height"], cam["width"]
    P = H * W
    S = gsr.Scene(scene)
    pins = {}
    for item in filter(None, args.pin.split(";")):
        name, vals = item.split("=")
        mode = {"pose_grad": gsr.GS_MODE_POSE_GRAD, "forward": gsr.GS_MODE_FORWARD}[name.strip()]
        pins[mode] = [int(x) for x in vals.split(",")]
        gsr.gs_scene_set_launch(S.handle, mode, [cam], *pins[mode])
    tgt = S.render(cam, T_ref)
    trgb, tdep = tgt["rgb"].clone(), tgt["depth"].clone()
    result = torch.zeros(8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    cam_c, pose_q = gsr.camera(cam), gsr.pose(T_q)
    out_f = S.alloc_outputs(cam, last_idx=False)
    out_fs = S.outputs_struct(out_f)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def grad_step():
        gsr.gs_render_pose_grad_async(S.handle, cam_c, pose_q, trgb.data_ptr(), tdep.data_ptr(), None, 0.1, None,
                                      result.data_ptr(), stream)

    def fwd_step():
        gsr.gs_render_async(S.handle, cam_c, pose_q, out_fs, stream)

    # size the workspace with one synchronous call, then check the async path
    S.render_pose_grad(cam, T_q, trgb, tdep)
    for _ in range(args.warmup):
        grad_step()
    st, n_rec, n_pairs = S.status()
    if st != 0:
        raise RuntimeError("workspace overflow in warm-up")

    def timed(fn, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        barrier(world)
        torch.cuda.synchronize()
        for a, b in ev:
            flush.zero_()
            a.record()
            fn()
            b.record()
        torch.cuda.synchronize()
        barrier(world)
        return float(np.mean([a.elapsed_time(b) for a, b in ev]))

    bus = None
    try:
        bus = torch.cuda.get_device_properties(torch.cuda.current_device()).pci_bus_id
    except AttributeError:
        pass
    clocks = ClockSampler(bus)
    clocks.start()
    # the default launch configuration, then the autotuner's for this call shape
    ms_grad_default = max_over_ranks(timed(grad_step, args.steps), world)

    def tune(mode):
        if mode in pins:  # pinned on the command line
            return {"best": gsr.gs_scene_get_launch(S.handle, mode, [cam]), "pinned": True}
        return gsr.gs_autotune(S.handle, mode, [cam], [T_q], reps=10)

    tune_grad = tune(gsr.GS_MODE_POSE_GRAD)
    for _ in range(args.warmup):
        grad_step()
    ms_grad = timed(grad_step, args.steps)
    ms_grad = max_over_ranks(ms_grad, world)
    st, _, _ = S.status()
    assert st == 0
    for _ in range(args.warmup):
        fwd_step()
    ms_fwd_default = max_over_ranks(timed(fwd_step, args.steps), world)
    tune_fwd = tune(gsr.GS_MODE_FORWARD)
    for _ in range(args.warmup):
        fwd_step()
    ms_fwd = max_over_ranks(timed(fwd_step, args.steps), world)

    # per-kernel device time over the same steps (events recorded by the library)
    gsr.gs_scene_set_timing(S.handle, True)
    gsr.gs_scene_kernel_times(S.handle)
    timed(grad_step, args.steps)
    kms, kn = gsr.gs_scene_kernel_times(S.handle)
    gsr.gs_scene_set_timing(S.handle, False)
    per_kernel = {name: kms[i] / kn[i] for i, name in enumerate(gsr.KERNEL_NAMES) if kn[i]}
    ts, _, _ = S.tile_lists(0, cam, n_pairs + 16)
    counts = np.diff(ts)
    tx, ty = (W + 15) // 16, (H + 15) // 16
    wt = np.minimum(16, W - 16 * np.arange(tx))
    ht = np.minimum(16, H - 16 * np.arange(ty))
    pair_pixels = int((counts * np.outer(ht, wt).reshape(-1)).sum())  # every pixel of every listed tile
    pk, pk_src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FMA = 2
    dom = max(per_kernel, key=per_kernel.get)
    kernels = {k: {"ms": v, "share": v / max(sum(per_kernel.values()), 1e-12)} for k, v in per_kernel.items()}
    # the step's work units, counted by the tangent pass itself: pairs blended,
    # and list entries examined before each pixel's stop (the definition's walk)
    blends, evals = gsr.gs_scene_work_counts(S.handle)
    if dom == "composite":
        flops = evals * FLOPS_PER_EVAL + blends * FLOPS_PER_BLEND
        ach = flops / (per_kernel[dom] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                "traffic": COMPOSITE_DRAM_BYTES, "kernel": "composite (tangent pass)",
                "work": "%d (pixel, Gaussian) evaluations x %d fp32 ops (skip path) + %d blended pairs x %d "
                        "(blend + six-direction tangent update)" % (evals, FLOPS_PER_EVAL, blends, FLOPS_PER_BLEND),
                "peak_source": "%d SMs x 128 fp32 lanes x 2 x %.0f MHz (%s max clock)" % (n_sm, sm_max, pk_src)}
    else:
        nsh = 48
        bytes_ = 1_000_000 * 16 + n_rec * (32 + 4 * nsh + 64)
        ach = bytes_ / (per_kernel[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                "traffic": None, "kernel": dom, "peak_source": pk_src}

    # the binning-side kernels against the HBM copy bandwidth, each on its algorithmic bytes
    # (their data mostly stays in the L2, so these fractions measure latency, not bandwidth)
    n_tiles = tx * ty
    alg_bytes = {"project": 16 * 1_000_000 + 32 * n_rec,       # means of all, covariances of the visible
                 "shade": n_rec * (48 + 4 * 48 + 64 + 4 * 48),  # record + SH in, record + pose Jacobian out
                 "scan_tiles": 12 * n_tiles,                     # counts in, offsets and cursors out
                 "scatter": 16 * n_rec + 8 * n_pairs,            # record bounds in, (depth, record) pairs out
                 "sort": 16 * n_pairs}                           # pairs in and out
    kernel_roofs = {k: {"bytes": b, "gbs": b / (per_kernel[k] * 1e-3) / 1e9,
                        "frac": b / (per_kernel[k] * 1e-3) / 1e9 / pk["hbm_gbs"]}
                    for k, b in alg_bytes.items() if per_kernel.get(k)}

    # end to end through the public API: pinned host targets -> device, synchronous call, result to host
    h_rgb = trgb.cpu().pin_memory()
    h_dep = tdep.cpu().pin_memory()

    def e2e_step():  # host targets in, (loss, gradient) out; the upload overlaps projection and binning
        return S.render_pose_grad_host(cam, T_q, h_rgb, h_dep)

    for _ in range(args.warmup):
        e2e_step()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, world)
    h2d = (h_rgb.numel() + h_dep.numel()) * 4

    # pose refinement (500k Gaussians, 960x540, 50 Adam iterations), single and 8 poses batched
    refine = None if args.no_refine else bench_refine(gsr, synth, torch)
    # batched vs single pose: 84 candidate views of mixed resolution in one graph launch
    batched = None
    if not args.no_batched:
        batched = bench_batched(gsr, synth, torch, flush, max(2, args.steps // 4), args.warmup)
    # large streamed scene: 6M Gaussians in 16 partitions, 8 poses through a 4-level pyramid
    with_oracle = rank == 0 and world == 1 and not args.no_cpu and not args.no_errors
    large_errors = []
    large = None if args.no_large else bench_large(gsr, synth, torch, large_errors if with_oracle else None)
    # error of every output and of the pose gradient against the fp64 oracle
    errors = None
    if with_oracle:
        errors = {"sample": "%d random pixels per view (fixed seed); pixels whose decisions the oracle flags as "
                            "near-ties are excluded from the image errors and weighted 0 in both gradients"
                            % ERR_PIXELS,
                  "aerial_1080p": view_errors(gsr, torch, S, scene, cam, T_ref, T_q, 1),
                  "large_pyramid": large_errors or None}
    # dense matching of rendered feature maps (PMM, Eq. 11) at 1920x1080: 32,400 x 32,400 similarities
    pmm = None
    if not args.no_pmm:
        pmm = bench_pmm(gsr, synth, torch, pk_for_pmm(), max(3, args.steps // 4), args.warmup,
                        with_oracle=rank == 0 and world == 1 and not args.no_cpu)
    # Algorithm 1 visibility check of all 1M Gaussians from the query pose
    vis = None
    if not args.no_vis:
        vis = bench_visibility(gsr, torch, S, scene, cam, T_q, flush, max(3, args.steps // 2), args.warmup,
                               with_oracle=rank == 0 and world == 1 and not args.no_cpu)
    # dense stage at 1080p: PMM -> PnP + RANSAC (Eq. 10), and three rounds with Algorithm 2
    dense = None
    if not args.no_dense:
        dense = bench_dense(gsr, synth, torch, max(3, args.steps // 2), args.warmup, pk_for_pmm(),
                            with_oracle=rank == 0 and world == 1 and not args.no_cpu)
    clk = clocks.stop()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(scene, cam, T_ref, T_q, args.cpu_seconds)

    launches_per_step = 7  # project, shade, scan, scatter, sort, tangent pass, fp64 reduction of its tile partials
    value = job_mpix_per_s(world, P, ms_grad)
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_grad, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "gaussians": 1_000_000, "width": W, "height": H, "sh_degree": 3,
                   "records": int(n_rec), "pairs": int(n_pairs), "evaluations": int(evals),
                   "pair_pixels": pair_pixels, "blended": int(blends),
                   "l2": "flushed (256 MB write) between timed steps, outside the timed events",
                   "parallelism": "replicas" if world > 1 else "single",
                   "launch": {"pose_grad": tune_grad["best"], "forward": tune_fwd["best"],
                              "note": "chosen by the library's autotuner (gs_autotune) for this call shape"}},
        "untuned": {"ms_per_step": ms_grad_default, "fwd_ms": ms_fwd_default,
                    "value": job_mpix_per_s(world, P, ms_grad_default),
                    "note": "the same steps under the default launch configuration"},
        "pose_grad_iters_per_s": world / (ms_grad * 1e-3),
        "fwd_mpix_s": job_mpix_per_s(world, P, ms_fwd), "fwd_ms": ms_fwd,
        "clocks": clk,
        "e2e": {"value": job_mpix_per_s(world, P, e2e_ms), "unit": "Mpix/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 7 * 8,
                "transfer": "pinned host targets read in place by the compositing pass over the CPU-GPU link; "
                            "(loss, gradient) copied back"},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof, "kernels": kernels, "kernel_rooflines": kernel_roofs,
        "refine": refine, "batched": batched, "large": large, "pmm": pmm, "visibility": vis, "dense": dense,
        "errors": errors,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    S.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def _pose_errors(T, T_ref):
    """Rotation angle of R R_ref^T with the trace clamp of the paper's Algorithm 2
    (degrees) and the distance between camera centres (metres)."""
    T, T_ref = np.asarray(T), np.asarray(T_ref)
    tr = float(np.clip(np.trace(T[:3, :3] @ T_ref[:3, :3].T), -1.0, 3.0))
    ang = math.degrees(math.acos((tr - 1.0) / 2.0))
    c = -T[:3, :3].T @ T[:3, 3]
    c_ref = -T_ref[:3, :3].T @ T_ref[:3, 3]
    return ang, float(np.linalg.norm(c - c_ref))


def bench_refine(gsr, synth, torch):
    scene, cam, T_gt, T_q = synth.refine_workload()
    S = gsr.Scene(scene)
    stream = torch.cuda.current_stream().cuda_stream
    tgt = S.render(cam, T_gt)
    tr, td = tgt["rgb"].clone(), tgt["depth"].clone()
    opts = gsr.gs_refine_defaults()
    warm = gsr.gs_refine_defaults()
    warm.iterations = 3
    gsr.gs_refine_pose(S.handle, gsr.camera(cam), gsr.pose(T_q), tr.data_ptr(), td.data_ptr(), None, warm, stream)
    torch.cuda.synchronize()
    p = gsr.pose(T_q)
    t0 = time.perf_counter()
    hist = gsr.gs_refine_pose(S.handle, gsr.camera(cam), p, tr.data_ptr(), td.data_ptr(), None, opts, stream)
    dt = time.perf_counter() - t0
    a0, d0 = _pose_errors(T_q, T_gt)
    a1, d1 = _pose_errors(gsr.pose_matrix(p), T_gt)
    single = {"iterations": opts.iterations, "iters_per_s": opts.iterations / dt, "ms_per_iter": dt * 1e3 / opts.iterations,
              "rot_err_deg": [a0, a1], "centre_err_m": [d0, d1], "loss": [float(hist[0]), float(hist[-1])]}
    # 8 query poses of the same scene: batched refinement vs one pose per launch
    g = synth.rng(11)
    refs = [synth.look_pose((g.uniform(400, 600), g.uniform(180, 220), g.uniform(280, 320)), g.uniform(-0.2, 0.2),
                            math.radians(g.uniform(25, 35))) for _ in range(8)]
    qs = [synth.perturb_pose(T, g, 2.0, 5.0) for T in refs]
    tg = []
    for T in refs:
        o = S.render(cam, T)
        tg.append((o["rgb"].clone(), o["depth"].clone()))
    it = 50
    o8 = gsr.gs_refine_defaults()
    o8.iterations = it
    cams = [gsr.camera(cam)] * 8
    w8 = gsr.gs_refine_defaults()
    w8.iterations = 2
    gsr.gs_refine_poses_batch(S.handle, cams, [gsr.pose(T) for T in qs], [a.data_ptr() for a, _ in tg],
                              [b.data_ptr() for _, b in tg], None, w8, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for T, (a, b) in zip(qs, tg):
        gsr.gs_refine_pose(S.handle, gsr.camera(cam), gsr.pose(T), a.data_ptr(), b.data_ptr(), None, o8, stream)
    t_single = time.perf_counter() - t0
    poses = [gsr.pose(T) for T in qs]
    t0 = time.perf_counter()
    gsr.gs_refine_poses_batch(S.handle, cams, poses, [a.data_ptr() for a, _ in tg], [b.data_ptr() for _, b in tg],
                              None, o8, stream)
    t_batch = time.perf_counter() - t0
    errs = [_pose_errors(gsr.pose_matrix(p), T) for p, T in zip(poses, refs)]
    S.close()
    return {"workload": "500k Gaussians SH3, 960x540 f=700, query 2 deg / 5 m off; Adam lr 1e-3 rad, 0.5 m",
            "single": single,
            "batched_8": {"views": 8, "iterations": it, "single_s": t_single, "batched_s": t_batch,
                          "speedup": t_single / t_batch, "pose_iters_per_s": 8 * it / t_batch,
                          "final_rot_err_deg_median": float(np.median([e[0] for e in errs])),
                          "final_centre_err_m_median": float(np.median([e[1] for e in errs])),
                          "final_rot_err_deg_max": max(e[0] for e in errs),
                          "final_centre_err_m_max": max(e[1] for e in errs),
                          "converged": int(sum(e[0] < 0.5 and e[1] < 1.25 for e in errs)),
                          "note": "photometric Adam from 2 deg / 5 m: a start outside the basin of the L1 loss "
                                  "does not converge (the batch equals the single-pose runs bit for bit)"}}


def bench_large(gsr, synth, torch, errors=None):
    """6M streamed Gaussians, 8 poses, 4-level pyramid of batched Adam refinement.
    errors: a list to receive view_errors() of the first pose at each level
    (the oracle's fp64 reference; None skips it)."""
    t0 = time.perf_counter()
    scene = synth.partitioned_scene(5, 4, 4, 375_000, cell_m=500.0, sh_degree=3, feat_dim=32,
                                    keep_f32=errors is not None)
    t_gen = time.perf_counter() - t0
    S = gsr.Scene(scene, stream_partitions=True)
    stream = torch.cuda.current_stream().cuda_stream
    g = synth.rng(12)
    refs = [synth.look_pose((g.uniform(700, 1300), g.uniform(700, 1300), g.uniform(250, 350)),
                            g.uniform(0, 2 * math.pi), math.radians(g.uniform(15, 35))) for _ in range(8)]
    qs = [synth.perturb_pose(T, g, 1.0, 2.0) for T in refs]
    if errors is not None:
        for level in range(4):
            cam = synth.camera(480 * 2 ** level, 270 * 2 ** level, 350.0 * 2 ** level)
            errors.append(view_errors(gsr, torch, S, scene, cam, refs[0], qs[0], 100 + level))
    del scene
    poses = [gsr.pose(T) for T in qs]
    start_err = [_pose_errors(gsr.pose_matrix(p), T) for p, T in zip(poses, refs)]
    levels = []
    for level in range(4):
        f = 350.0 * 2 ** level
        cam = synth.camera(480 * 2 ** level, 270 * 2 ** level, f)
        outs = [S.alloc_outputs(cam, feat_dim=32, last_idx=False) for _ in refs]
        b0 = S.stream_stats()[0]
        S.render_batch([cam] * 8, refs, outs)  # targets at this level (with the feature maps)
        tr = [o["rgb"] for o in outs]
        td = [o["depth"] for o in outs]
        opts = gsr.gs_refine_defaults()
        opts.iterations = 20
        # the autotuner's configuration for this level's 8-view pose-gradient batch
        tune = gsr.gs_autotune(S.handle, gsr.GS_MODE_POSE_GRAD, [cam] * 8, [gsr.pose_matrix(p) for p in poses],
                               reps=3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist = gsr.gs_refine_poses_batch(S.handle, [gsr.camera(cam)] * 8, poses, [a.data_ptr() for a in tr],
                                         [b.data_ptr() for b in td], None, opts, stream)
        dt = time.perf_counter() - t0
        b1, res, act = S.stream_stats()
        errs = [_pose_errors(gsr.pose_matrix(p), T) for p, T in zip(poses, refs)]
        levels.append({"width": cam["width"], "height": cam["height"], "iterations": 20, "seconds": dt,
                       "launch": tune,
                       "pose_iters_per_s": 8 * 20 / dt, "mpix_per_s": 8 * 20 * cam["width"] * cam["height"] / dt / 1e6,
                       "h2d_bytes": b1 - b0, "resident_partitions": res,
                       "loss_first_last": [float(hist[:, 0].mean()), float(hist[:, -1].mean())],
                       "rot_err_deg_median": float(np.median([e[0] for e in errs])),
                       "centre_err_m_median": float(np.median([e[1] for e in errs]))})
        del outs, tr, td
    S.close()
    return {"workload": "6M Gaussians (16 partitions of 375k, 4x4 cells of 500 m), SH3 + 32 BF16 features, "
                        "streamed; 8 query poses 1 deg / 2 m off; 4-level pyramid, 20 batched Adam iterations each",
            "generation_s": t_gen,
            "start_rot_err_deg_median": float(np.median([e[0] for e in start_err])),
            "start_centre_err_m_median": float(np.median([e[1] for e in start_err])),
            "levels": levels}


ERR_PIXELS = 20_000


def _err_stats(d):
    d = np.abs(np.asarray(d, np.float64))
    return {"max_abs": float(d.max()) if d.size else 0.0, "rms": float(np.sqrt((d ** 2).mean())) if d.size else 0.0}


def view_errors(gsr, torch, S, scene, cam, T_ref, T_q, seed):
    """Max-abs and RMS error of every output of the library's render at T_q
    (rgb, depth, alpha, final T and, with features, the 32 feature channels)
    against the fp64 oracle on ERR_PIXELS random pixels, and of the pose
    gradient of the L1 loss against targets rendered by the library at T_ref,
    component by component. With features, the error of their bf16 storage
    (the oracle blending the unrounded binary32 vectors against the bf16 ones)
    is reported apart from the fp32 blending error."""
    from oracle import oracle as O
    O.build()
    n_thr = os.cpu_count() or 1
    H, W = cam["height"], cam["width"]
    feats = scene.get("feats_bf16") is not None
    tgt = S.render(cam, T_ref, S.alloc_outputs(cam, last_idx=False))
    trgb, tdep = tgt["rgb"].contiguous(), tgt["depth"].contiguous()
    out = S.render(cam, T_q, S.alloc_outputs(cam, feat_dim=32 if feats else 0, last_idx=False))
    gpu = {k: v.cpu().numpy().reshape(v.shape[0] if v.dim() == 3 else 1, H * W).T for k, v in out.items()}
    pix = np.sort(np.random.default_rng(seed).choice(H * W, min(ERR_PIXELS, H * W), replace=False))
    mask = np.zeros((H, W), np.float32)
    mask.reshape(-1)[pix] = 1.0
    trgb_h, tdep_h = trgb.cpu().numpy(), tdep.cpu().numpy()
    osc = O.OracleScene(scene)
    t0 = time.perf_counter()
    orc = O.render(osc, cam, T_q, geom64=True, pixels=pix, target_rgb=trgb_h, target_depth=tdep_h,
                   pixel_weight=mask, n_threads=n_thr)
    ok = (orc["flags"] & O.TIE_IMAGE) == 0
    res = {"width": W, "height": H, "pixels": int(len(pix)), "excluded_near_ties": int((~ok).sum()), "outputs": {}}
    for k in ("rgb", "depth", "alpha", "final_T") + (("feats",) if feats else ()):
        g = gpu[k][pix][ok]
        o = np.asarray(orc[k]).reshape(len(pix), -1)[ok]
        res["outputs"][k] = dict(_err_stats(g - o), oracle_max=float(np.abs(o).max()))
    if feats:  # bf16 storage error, apart from the blending error above
        o32 = O.render(O.OracleScene(scene, unrounded_feats=True), cam, T_q, geom64=True, pixels=pix[ok],
                       n_threads=n_thr)
        res["outputs"]["feats_bf16_storage"] = dict(_err_stats(orc["feats"][ok] - o32["feats"]),
                                                    note="oracle with bf16 features minus oracle with the "
                                                         "unrounded binary32 features")
    # pose gradient: pixels of the sample without any near-tie decision
    w = np.zeros((H, W), np.float32)
    w.reshape(-1)[pix[orc["flags"] == 0]] = 1.0
    og = O.render(osc, cam, T_q, geom64=True, want_grad=True, pixels=pix, target_rgb=trgb_h, target_depth=tdep_h,
                  pixel_weight=w, n_threads=n_thr, want_feats=False)
    res["oracle_s"] = time.perf_counter() - t0
    loss, grad = S.render_pose_grad(cam, T_q, trgb, tdep, torch.from_numpy(w).cuda())
    og_g = np.asarray(og["grad"], np.float64)
    comp = []
    for k, name in enumerate(("rho_x", "rho_y", "rho_z", "phi_x", "phi_y", "phi_z")):
        e = abs(float(grad[k]) - og_g[k])
        comp.append({"component": name, "gpu": float(grad[k]), "oracle": float(og_g[k]), "abs_err": e,
                     "rel_err": e / max(abs(og_g[k]), 1e-300)})
    blocks = []
    for sl in (slice(0, 3), slice(3, 6)):
        blocks.append(float(np.linalg.norm(np.asarray(grad[sl]) - og_g[sl]) / max(np.linalg.norm(og_g[sl]), 1e-300)))
    res["gradient"] = {"pixels": int(w.sum()), "loss_rel_err": abs(loss - og["loss"]) / max(abs(og["loss"]), 1e-300),
                       "components": comp, "block_rel_err": {"rho": blocks[0], "phi": blocks[1]}}
    return res


def pk_for_pmm():
    pk, src = peaks()
    return pk, src


def bench_pmm(gsr, synth, torch, pk_src, steps, warmup, with_oracle=False):
    """PMM (Sec. 3.4, Eq. 11) of the query-pose feature map against the reference
    one, both rendered by the library from 1M Gaussians with 32 BF16 channels.
    With the oracle: the coarse decisions of the fp64 definition on the same
    maps at 960x536, against the library's and against a single-bf16
    contraction's."""
    pk, src = pk_src
    scene = synth.aerial_scene(2, 1_000_000, feat_dim=32)
    cam = synth.aerial_camera()
    T_ref = synth.aerial_pose()
    T_q = synth.perturb_pose(T_ref, synth.rng(100), 2.0, 5.0)
    S = gsr.Scene(scene)
    maps = []
    for T in (T_q, T_ref):
        o = S.alloc_outputs(cam, feat_dim=32, last_idx=False)
        S.render(cam, T, o)
        maps.append(o["feats"].contiguous())
    S.close()
    H, W = cam["height"], cam["width"]
    M = gsr.Matcher(H, W)
    for _ in range(warmup):
        res = M.match(maps[0], maps[1])
    # the C-ABI call alone: the binding's copies of the matcher's device outputs stay outside the events
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record()
        M.match_raw(maps[0], maps[1])
        b.record()
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    res = M.match(maps[0], maps[1])
    M.close()
    n = (H // 8) * (W // 8)
    sims = float(n) * n
    mma_flops = 3 * 2 * 2 * 32 * sims  # three split products, two passes over the tiles, K = 32
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    mufu_peak = sm * 16 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6  # exp2 per second (16 per SM per clock)
    decisions = pmm_decisions(gsr, synth, torch, scene, T_ref, T_q) if with_oracle else None
    return {"workload": "PMM of 1920x1080 32-channel feature maps rendered from 1M Gaussians (query 2 deg / 5 m "
                        "off the reference): 8x8 coarse cells, tau 0.1, coarse MNN + 8x8-window fine MNN",
            "coarse_precision": "split bf16 (hi + lo) operands, hi.hi + lo.hi + hi.lo, fp32 accumulation",
            "decisions_vs_fp64_definition": decisions,
            "cells": n, "similarities": int(sims), "ms": ms, "coarse_matches": int(res["coarse"].shape[0]),
            "fine_matches": int(res["fine"].shape[0]),
            "similarities_per_s": sims / (ms * 1e-3),
            "tensor": {"flops": mma_flops, "achieved_tflops": mma_flops / (ms * 1e-3) / 1e12,
                       "peak_tflops": pk.get("bf16_tflops"), "frac": mma_flops / (ms * 1e-3) / 1e12 /
                       float(pk.get("bf16_tflops", 1965.2)), "peak_source": src,
                       "note": "K = 32: the contraction is small; the epilogue (exp, reductions, argmax) bounds"},
            "exp": {"count": int(sims), "achieved_per_s": sims / (ms * 1e-3), "mufu_peak_per_s": mufu_peak,
                    "frac": sims / (ms * 1e-3) / mufu_peak}}


def pmm_decisions(gsr, synth, torch, scene, T_ref, T_q):
    """Coarse decisions of the library against the fp64 definition of Eq. 11 (the
    oracle) on 960x536 feature maps rendered by the library: the fraction of
    decisions clear of ties, the library's changes among those (must be 0), and
    what a single-bf16 contraction (the oracle's precision layer) would change."""
    from oracle import pmm as OP
    cam = synth.aerial_camera(960, 536, 700.0)  # both sides multiples of the coarse ratio 8
    S = gsr.Scene(scene)
    maps = []
    for T in (T_q, T_ref):
        o = S.alloc_outputs(cam, feat_dim=32, last_idx=False)
        S.render(cam, T, o)
        maps.append(o["feats"].contiguous())
    S.close()
    M = gsr.Matcher(536, 960)
    g = {k: v.cpu().numpy() for k, v in M.match(maps[0], maps[1]).items()}
    M.close()
    Fq, Fr = (m.cpu().numpy() for m in maps)
    t0 = time.perf_counter()
    d = OP.coarse_pmm(Fq, Fr)
    dt = time.perf_counter() - t0
    b = OP.coarse_pmm_bf16(Fq, Fr)
    rok, cok = ~d["row_flag"], ~d["col_flag"]
    gm = {tuple(x) for x in g["coarse"].tolist()}
    dm = {tuple(x) for x in d["matches"].tolist()}
    clear = lambda ij: rok[ij[0]] and cok[ij[1]]
    return {"maps": "960x536 (8,040 coarse cells), library renders of the same scene and poses",
            "clear_of_ties": {"rows": float(rok.mean()), "cols": float(cok.mean()), "tie_gap_logP": OP.TIE_GAP},
            "library_vs_definition_clear": {
                "rows": float((g["row_best"][rok] != d["row_best"][rok]).mean()),
                "cols": float((g["col_best"][cok] != d["col_best"][cok]).mean()),
                "matches": len({x for x in gm if clear(x)} ^ {x for x in dm if clear(x)}) / max(1, len(dm))},
            "single_bf16_layer_vs_definition": OP.decision_changes(b, d),
            "oracle_s": dt}


def bench_visibility(gsr, torch, S, scene, cam, T, flush, steps, warmup, with_oracle):
    """Render-gradient visibility check (Sec. 3.2, Algorithm 1) of every Gaussian
    of the headline scene from the query pose, through gs_visibility."""
    n = S.n
    for _ in range(warmup):
        r = S.visibility(cam, T)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for a, b in ev:
        flush.zero_()
        a.record()
        r = S.visibility(cam, T)
        b.record()
    torch.cuda.synchronize()
    wall_ms = (time.perf_counter() - t0) * 1e3 / steps
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    gsr.gs_scene_set_timing(S.handle, True)
    gsr.gs_scene_kernel_times(S.handle)
    for _ in range(steps):
        flush.zero_()
        S.visibility(cam, T)
    kms, kn = gsr.gs_scene_kernel_times(S.handle)
    gsr.gs_scene_set_timing(S.handle, False)
    per_kernel = {name: kms[i] / kn[i] for i, name in enumerate(gsr.KERNEL_NAMES) if kn[i]}
    blends, evals = gsr.gs_scene_work_counts(S.handle)
    pk, pk_src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    t_bw = per_kernel["vis_backward"]
    flops = evals * FLOPS_PER_EVAL + blends * FLOPS_PER_VIS_BLEND
    ach = flops / (t_bw * 1e-3) / 1e12
    mask = r["mask"].cpu().numpy()
    out = {"workload": "Algorithm 1 visibility of all 1M Gaussians (aerial SH3) at 1920x1080 from the query pose: "
                       "forward render, reverse pass of sum(RGB), mean gradients, in-image test, compaction",
           "gaussians": n, "kept": int(r["n_visible"]), "m_r": int(((mask & 2) != 0).sum()),
           "m_i": int(((mask & 4) != 0).sum()), "ms": ms, "wall_ms": wall_ms,
           "gaussians_per_s": n / (ms * 1e-3),
           "kernels": {k: {"ms": v, "share": v / max(sum(per_kernel.values()), 1e-12)} for k, v in per_kernel.items()},
           "roofline": {"bound": "alu", "kernel": "vis_backward (reverse pass, accumulator zeroing included)",
                        "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                        "traffic": VIS_BACKWARD_DRAM_BYTES,
                        "work": "%d (pixel, Gaussian) evaluations x %d + %d blended pairs x %d (reverse blend, "
                                "monomial sums, warp reduction)" % (evals, FLOPS_PER_EVAL, blends,
                                                                    FLOPS_PER_VIS_BLEND),
                        "peak_source": "%d SMs x 128 fp32 lanes x 2 x %.0f MHz (%s max clock)"
                                       % (n_sm, sm_max, pk_src)},
           "l2": "flushed (256 MB write) between timed calls, outside the timed events"}
    if with_oracle:
        from oracle import oracle as O
        O.build()
        n_thr = os.cpu_count() or 1
        keep = np.nonzero(mask & 2)[0]
        sample = np.sort(np.random.default_rng(1).choice(keep, min(16, len(keep)), replace=False))
        t0 = time.perf_counter()
        O.visibility(scene, cam, T, n_threads=n_thr, gids=sample)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": len(sample) / dt, "unit": "Gaussians/s", "cores": n_thr, "kind": "oracle",
                               "sample": "fp64 oracle mean gradient (forward mode, one Gaussian at a time over its "
                                         "tile rectangle) of %d Gaussians with M^r, %.2f s" % (len(sample), dt)}
    return out


def bench_dense(gsr, synth, torch, steps, warmup, pk_src, with_oracle):
    """The dense stage of Sec. 3.4 at 1920x1080 on 1M Gaussians with 32 BF16
    features. The query image's feature map is the library's render at the
    query pose; the render pose is 2 deg / 5 m away. One round: PMM of the
    query features against the render's, PnP + RANSAC (128 P3P samples) on the
    fine matches lifted through the rendered depth. Then gs_dense_localize: three
    such rounds from the render pose and Algorithm 2's check."""
    pk, src = pk_src
    scene = synth.aerial_scene(2, 1_000_000, feat_dim=32)
    cam = synth.aerial_camera()
    T_r = synth.aerial_pose()
    T_q = synth.perturb_pose(T_r, synth.rng(100), 2.0, 5.0)
    H, W = cam["height"], cam["width"]
    S = gsr.Scene(scene)
    oq = S.alloc_outputs(cam, feat_dim=32, last_idx=False)
    S.render(cam, T_q, oq)
    Fq = oq["feats"].contiguous()
    orr = S.alloc_outputs(cam, feat_dim=32, last_idx=False)
    S.render(cam, T_r, orr)
    M = gsr.Matcher(H, W)
    res = M.match(Fq, orr["feats"].contiguous())
    fine = res["fine"].contiguous()
    n_hyp = 128
    words_np = np.random.default_rng(5).integers(0, 2 ** 32, (3, n_hyp, 3), dtype=np.uint64).astype(np.uint32)
    words = torch.from_numpy(words_np.view(np.int32)).cuda()
    P = gsr.PnP(H * W, n_hyp)
    depth, alpha = orr["depth"].contiguous(), orr["alpha"].contiguous()
    for _ in range(warmup):
        r = P.solve(cam, T_r, depth, alpha, fine, words[0])
    # the C-ABI call alone: the binding's copies of the solver's device outputs stay outside the events
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record()
        P.solve_raw(cam, T_r, depth, alpha, fine, words[0])
        b.record()
    torch.cuda.synchronize()
    ms_pnp = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    r = P.solve(cam, T_r, depth, alpha, fine, words[0])
    gsr.gs_pnp_set_timing(P.handle, True)
    gsr.gs_pnp_phase_times(P.handle)
    for _ in range(steps):
        P.solve(cam, T_r, depth, alpha, fine, words[0])
    ph_ms, ph_n = gsr.gs_pnp_phase_times(P.handle)
    gsr.gs_pnp_set_timing(P.handle, False)
    phases = {k: float(ph_ms[i] / max(ph_n, 1)) for i, k in enumerate(gsr.PNP_PHASES)}
    n_sol = int((r["hyp_counts"] >= 0).sum().item())
    pairs = n_sol * int(r["n_valid"])
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    ach = pairs * FLOPS_PER_PNP_PAIR / (phases["score"] * 1e-3) / 1e12
    err = _pose_errors(r["T"], T_q)
    # Algorithm 2: three rounds from the render pose
    loc = gsr.dense_localize(S, M, P, cam, T_r, Fq, words)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(2, steps // 2)):
        loc = gsr.dense_localize(S, M, P, cam, T_r, Fq, words)
    torch.cuda.synchronize()
    ms_loc = (time.perf_counter() - t0) * 1e3 / max(2, steps // 2)
    out = {"workload": "dense stage at 1920x1080, 1M Gaussians with 32-channel BF16 features; query features "
                       "rendered at a pose 2 deg / 5 m from the render pose; PMM fine matches -> PnP + RANSAC "
                       "(128 P3P samples, tau 2 px, 5 Gauss-Newton steps); Algorithm 2 over 3 rounds",
           "fine_matches": int(fine.shape[0]), "with_depth": int(r["n_valid"]), "inliers": int(r["n_inliers"]),
           "solutions": n_sol, "pnp_ms": ms_pnp, "pnp_phases_ms": phases,
           "pose_error_after_one_round": {"rot_deg": err[0], "centre_m": err[1]},
           "start_error": dict(zip(("rot_deg", "centre_m"), _pose_errors(T_r, T_q))),
           "roofline": {"bound": "alu", "kernel": "k_pnp_score (every P3P solution against every match)",
                        "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                        "traffic": PNP_SCORE_DRAM_BYTES,
                        "work": "%d solutions x %d matches x %d fp32 ops" % (n_sol, int(r["n_valid"]),
                                                                         FLOPS_PER_PNP_PAIR),
                        "peak_source": "%d SMs x 128 fp32 lanes x 2 x %.0f MHz (%s max clock)"
                                       % (n_sm, sm_max, src)},
           "algorithm2": {"ms_per_localisation": ms_loc, "rounds": loc["n_rounds"], "reliable": loc["reliable"],
                          "angles_deg": loc["angle_deg"], "matches": loc["n_matches"], "inliers": loc["n_inliers"],
                          "final_error": dict(zip(("rot_deg", "centre_m"), _pose_errors(loc["T"], T_q)))}}
    if with_oracle:
        from oracle import oracle as O
        from oracle import pnp as OPn
        O.build()
        m_np = fine.cpu().numpy()
        d_np, a_np = depth.cpu().numpy(), alpha.cpu().numpy()
        n_s = 8
        t0 = time.perf_counter()
        OPn.pnp_ransac(d_np, a_np, cam, T_r, m_np, words_np[0][:n_s], refine_iters=2)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": n_s / dt, "unit": "hypotheses/s (lift + P3P + scoring, 2 GN steps)",
                               "cores": os.cpu_count() or 1, "kind": "oracle",
                               "sample": "fp64 oracle PnP + RANSAC with %d of the 128 samples on all %d fine matches, "
                                         "%.2f s" % (n_s, int(fine.shape[0]), dt)}
    P.close()
    M.close()
    S.close()
    return out


FLOPS_PER_FEAT_BLEND = 12 + 2 * 32  # a blend of the forward pass: blend 12, then 32 feature FMAs


def fp32_peak_tflops(torch):
    pk, src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    return n_sm * 128 * 2 * sm_max * 1e6 / 1e12, "%d SMs x 128 fp32 lanes x 2 x %.0f MHz (%s max clock)" % (
        n_sm, sm_max, src)


def kernel_times(gsr, S, fn, reps):
    """Per-kernel device times (ms per call) of `fn` from the library's own
    events (the passes then run in order, without the shading stream)."""
    gsr.gs_scene_set_timing(S.handle, True)
    gsr.gs_scene_kernel_times(S.handle)
    for _ in range(reps):
        fn()
    kms, kn = gsr.gs_scene_kernel_times(S.handle)
    gsr.gs_scene_set_timing(S.handle, False)
    per = {name: kms[i] / reps for i, name in enumerate(gsr.KERNEL_NAMES) if kn[i]}
    tot = max(sum(per.values()), 1e-12)
    return {k: {"ms": v, "share": v / tot} for k, v in per.items()}


def bench_batched(gsr, synth, torch, flush, steps, warmup, n_views=None):
    """84 candidate poses at three pyramid levels (64 @ 480x270, 16 @ 960x540,
    4 @ 1920x1080), 2M Gaussians with 32 BF16 features: one graph launch
    against 84 single-view launches, forward (with the feature map) and pose
    gradient, under the default launch configurations and after the
    autotuner has picked one per call shape (the batch, and each level's
    single view). Per-kernel times and the dominant kernel's roofline."""
    scene = synth.partitioned_scene(4, 2, 2, 500_000, sh_degree=3, feat_dim=32)
    cams, poses = synth.batched_views()
    if n_views:
        cams, poses = cams[:n_views], poses[:n_views]
    S = gsr.Scene(scene)
    outs = [S.alloc_outputs(c, feat_dim=32, last_idx=False) for c in cams]
    structs = [S.outputs_struct(o) for o in outs]
    stream = torch.cuda.current_stream().cuda_stream
    S.render_batch(cams, poses, outs)  # synchronous: sizes the workspace
    # pose-gradient targets: the rendered views; queries 1 deg / 1 m away
    tg = [(o["rgb"].clone(), o["depth"].clone()) for o in outs]
    qs = [synth.perturb_pose(T, synth.rng(500 + k), 1.0, 1.0) for k, T in enumerate(poses)]
    loss, grad = S.render_pose_grad_batch(cams, qs, [a for a, _ in tg], [b for _, b in tg])  # sizes the workspace
    q_blends, q_evals = gsr.gs_scene_work_counts(S.handle)
    # the forward pass walks the same lists as a pose gradient at the same poses
    S.render_pose_grad_batch(cams, poses, [a for a, _ in tg], [b for _, b in tg])
    f_blends, f_evals = gsr.gs_scene_work_counts(S.handle)
    _, n_rec, n_pairs = S.status()
    S.reserve(int(n_rec * 1.2) + 1024, int(n_pairs * 1.2) + 4096)
    cc = [gsr.camera(c) for c in cams]
    pp = [gsr.pose(T) for T in poses]
    qq = [gsr.pose(T) for T in qs]
    res_single = torch.zeros((len(cams), 8), dtype=torch.float64, device="cuda")
    res_batch = torch.zeros((len(cams), 8), dtype=torch.float64, device="cuda")

    def single():
        for c, p, o in zip(cc, pp, structs):
            gsr.gs_render_async(S.handle, c, p, o, stream)

    def batch():
        gsr.gs_render_batch(S.handle, cc, pp, structs, gsr.GS_BATCH_GRAPH, stream)

    def single_grad():
        for k, (c, p, (a, b)) in enumerate(zip(cc, qq, tg)):
            gsr.gs_render_pose_grad_async(S.handle, c, p, a.data_ptr(), b.data_ptr(), None, 0.1, None,
                                          res_single[k].data_ptr(), stream)

    def batch_grad():
        gsr.gs_render_pose_grad_batch(S.handle, cc, qq, [a.data_ptr() for a, _ in tg], [b.data_ptr() for _, b in tg],
                                      None, 0.1, None, res_batch.data_ptr(), gsr.GS_BATCH_GRAPH, stream)

    def time_all():
        res = {}
        for name, fn in (("single", single), ("batched", batch), ("single_grad", single_grad),
                         ("batched_grad", batch_grad)):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            st = S.status()[0]
            assert st == 0, "batched workspace overflow"
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, b in ev:
                flush.zero_()
                a.record()
                fn()
                b.record()
            torch.cuda.synchronize()
            res[name] = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        torch.testing.assert_close(res_single, res_batch, rtol=0, atol=0)
        return res

    px = sum(c["width"] * c["height"] for c in cams)

    def summary(res):
        return {"forward": {"single_ms": res["single"], "batched_ms": res["batched"],
                            "single_mpix_s": px / (res["single"] * 1e-3) / 1e6,
                            "batched_mpix_s": px / (res["batched"] * 1e-3) / 1e6,
                            "speedup": res["single"] / res["batched"]},
                "pose_grad": {"single_ms": res["single_grad"], "batched_ms": res["batched_grad"],
                              "single_pose_iters_per_s": len(cams) / (res["single_grad"] * 1e-3),
                              "batched_pose_iters_per_s": len(cams) / (res["batched_grad"] * 1e-3),
                              "speedup": res["single_grad"] / res["batched_grad"]}}

    default = summary(time_all())
    # the autotuner, per call shape: the 84-view batch and each level's single view
    tuning = {}
    levels = sorted({(c["width"], c["height"]) for c in cams})
    for mode, name in ((gsr.GS_MODE_FEATURES, "forward"), (gsr.GS_MODE_POSE_GRAD, "pose_grad")):
        tp = qs if mode == gsr.GS_MODE_POSE_GRAD else poses
        r = gsr.gs_autotune(S.handle, mode, cams, tp, reps=5)
        tuning[name] = {"batch": r}
        for (w, h) in levels:
            k = next(i for i, c in enumerate(cams) if (c["width"], c["height"]) == (w, h))
            tuning[name]["%dx%d" % (w, h)] = gsr.gs_autotune(S.handle, mode, [cams[k]], [tp[k]], reps=5)
    tuned = summary(time_all())
    # per-kernel device times of one batch call (library events, non-graph, passes in order)
    kf = kernel_times(gsr, S, lambda: S.render_batch(cams, poses, outs), 3)
    kg = kernel_times(gsr, S, lambda: S.render_pose_grad_batch(cams, qs, [a for a, _ in tg], [b for _, b in tg]), 3)
    peak, peak_src = fp32_peak_tflops(torch)

    def roof(kern, evals, blends, per_blend, what):
        t = kern["composite"]["ms"]
        fl = evals * FLOPS_PER_EVAL + blends * per_blend
        ach = fl / (t * 1e-3) / 1e12
        return {"bound": "alu", "kernel": what, "ms": t, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "peak_source": peak_src,
                "work": "%d list entries examined before the stop x %d + %d blended pairs x %d"
                        % (evals, FLOPS_PER_EVAL, blends, per_blend)}

    S.close()
    out = {"views": len(cams), "gaussians": 2_000_000, "feat_dim": 32, "mpix": px / 1e6,
           "outputs": "rgb, depth, alpha, T, 32 features", "default_launch": default, "tuned": tuned,
           "tuning": tuning,
           "kernels": {"forward": kf, "pose_grad": kg},
           "roofline": {"forward": roof(kf, f_evals, f_blends, FLOPS_PER_FEAT_BLEND,
                                        "composite, forward with the 32-channel feature map"),
                        "pose_grad": roof(kg, q_evals, q_blends, FLOPS_PER_BLEND, "composite, tangent pass")},
           "records": int(n_rec), "pairs": int(n_pairs)}
    out.update(tuned)
    return out


if __name__ == "__main__":
    main()
