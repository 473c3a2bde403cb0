#!/usr/bin/env python
"""Frame-rate benchmark of the LODGE render path on one node.

Workload: the outdoor LOD scene (16M / 4M / 1M / 250k Gaussians over a 1 km x
1 km heightfield, 16 x 16 chunk grid, SH degree 3, fp32 attributes) and a
300-pose street-level trajectory at 1920 x 1080.  A step renders
--poses-per-step consecutive poses (400 by default, wrapping around the
trajectory) in LOD+chunk mode with opacity blending (the paper's method)
through one render call, whose frames take turns on eight streams; value =
frames/s over all ranks.  Inputs are resident in HBM before timing (5.0 GB
scene, larger than L2, no flush between steps).  Reported beside it:
  * the same poses at full detail (every level-0 Gaussian) on the same GPU,
    and the speedup;
  * the latency and per-stage device times of single frames, the paper's
    timing protocol (median of 7 renders per pose), the compositing's
    roofline;
  * end to end through the host-buffer call over the same steps;
  * the oracle's frame rate on the host cores (cpu_baseline);
  * the large scene's 64-camera 4K call, a fine-tuning step of one level,
    and a serving sweep over four streamed scenes under a 60 GB budget.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lodge|reference]

Under torchrun (N > 1) every rank renders its own trajectory (weak scaling,
no data-path collective); the barrier and a max over ranks bracket the timed
region.  --impl reference times the CPU oracle on the same workload (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p frames/s, LOD+chunk vs full-detail 3DGS (same GPU); p50/p99 serve latency"
UNIT = "frames/s"

# stages of lodge_profile, in order
STAGES = ["select", "union", "project", "depth_sort", "emit", "tile_sort", "ranges", "blend"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["lodge", "reference"], default="lodge")
    ap.add_argument("--scale", type=float, default=1.0, help="scene size factor (1.0 = full)")
    ap.add_argument("--n-poses", type=int, default=300)
    ap.add_argument("--poses-per-step", type=int, default=400,
                    help="consecutive poses per render call (one step), wrapping around the "
                         "300-pose trajectory; 400 keeps the 20 timed steps above one second")
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--full-steps", type=int, default=None)
    ap.add_argument("--per-frame-calls", action="store_true",
                    help="one render call per pose instead of one per step")
    ap.add_argument("--cpu-budget-s", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--bin-log2", type=int, default=None,
                    help="key lists per bin of 2^k x 2^k tiles (default: the library's)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="duration of the serving run at --serve-rate (step mode)")
    ap.add_argument("--serve-warmup-s", type=float, default=5.0)
    ap.add_argument("--serve-slot-seconds", type=float, default=10.0,
                    help="duration of the slot-worker serving run")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large scene (60M level-0 Gaussians, 64 cameras at 4K)")
    ap.add_argument("--no-finetune", action="store_true",
                    help="skip the fine-tuning step (2M Gaussians, 32 views at 1280x720)")
    ap.add_argument("--finetune-steps", type=int, default=3)
    ap.add_argument("--no-next", action="store_true",
                    help="skip the threshold search, importance, build-loop and K-means timings")
    ap.add_argument("--large-scale", type=float, default=1.0)
    ap.add_argument("--serve-batch", type=int, default=16,
                    help="frames per step of the batched serving run")
    ap.add_argument("--serve-budget-gb", type=float, default=60.0)
    ap.add_argument("--serve-scale", type=float, default=1.0,
                    help="scene size factor of the serving scenes (1.0 = 2M/8M/16M/30M)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# multi-rank protocol (weak scaling: every rank renders its own trajectory)
def rank_trajectory_seed(seed: int, rank: int, world: int) -> int:
    """Trajectory seed of a rank: rank 0 keeps the base trajectory at N = 1."""
    return seed if world == 1 else seed + 1000 * rank


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value over ranks (the slowest rank bounds the job)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(frames_per_rank: int, world: int, t_max: float) -> float:
    """Whole-job frames/s: every rank's frames over the slowest rank's time."""
    return frames_per_rank * world / t_max


def timed_region(run, world: int, sync=None, clock=None, device=None):
    """Barrier, sync, run(), sync, barrier; returns the max over ranks of
    the time `clock` measured (default: host perf_counter around run)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if sync:
        sync()
    if clock is None:
        t0 = time.perf_counter()
        run()
        if sync:
            sync()
        t = time.perf_counter() - t0
    else:
        t = clock(run)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    return max_over_ranks(t, world, device)


# ---------------------------------------------------------------------------
def stage_bytes(stage: str, prof: dict) -> float:
    """Algorithmic bytes of one stage summed over the profiled frames."""
    a, v, k = prof["active"], prof["visible"], prof["keys"]
    if stage == "project":
        # list entry + means per active Gaussian; scale/opacity, quaternion and
        # 48 SH coefficients per visible Gaussian; 56 B of records written
        return a * (4 + 12) + v * (16 + 16 + 192 + 56)
    # one key per (record, bin): bins are tiles or squares of 2^k tiles.  Keys
    # of frames whose (bin, record) pair fits one word are written and sorted
    # as single 4 B words; the others as a 4 B key plus a 4 B value
    bk = prof.get("bin_keys", k)
    kp = prof.get("packed_keys", 0)
    if stage == "depth_sort":
        return v * (4 * 16)              # 4 passes of read/write key+value (digits counted by the projection)
    if stage == "emit":
        # fused emission: read the record id and its rect (12 B per visible),
        # write 4 or 8 B per key
        return v * 12 + kp * 4 + (bk - kp) * 8
    if stage == "tile_sort":
        # every pass (8 bits of the bin id each) reads and writes every key (and value)
        passes = prof.get("bin_sort_passes", 2 * prof["frames"]) / max(prof["frames"], 1)
        return (kp * 8 + (bk - kp) * 16) * passes
    if stage == "ranges":
        return bk * 4
    return 0.0


def measured_traffic(kernel_stage: str, units_per_launch: float):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary (profiles/traffic_*.txt), scaled to this run's units per launch
    where the summary gives bytes per unit; None if there is no summary for
    it or its kernel source changed since."""
    import hashlib
    files = {"blend": "traffic_blend_kernel.txt"}
    f = files.get(kernel_stage)
    if f is None:
        return None
    path = os.path.join(ROOT, "profiles", f)
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#") and "=" in line:
            k, v = line.split("=", 1)
            kv[k] = v
    src = os.path.join(ROOT, kv.get("source", ""))
    if not os.path.exists(src):
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != kv.get("source_sha256_16"):
        return None
    if "dram_bytes_per_launch" in kv:
        return float(kv["dram_bytes_per_launch"])
    return float(kv["dram_bytes_per_key"]) * units_per_launch


def run_lodge(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2505_23158_gb300 import build, synth
    from paper_2505_23158_gb300.api import CHUNK_BLEND, FULL, Lodge

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    t0 = time.time()
    scene, cams = synth.workload_outdoor(seed=args.seed, n_poses=args.n_poses, scale=args.scale,
                                         width=args.width, height_px=args.height)
    if world > 1:
        # weak scaling: every rank walks its own seeded trajectory of the same scene
        cams = synth.outdoor_trajectory(scene, seed=rank_trajectory_seed(args.seed, rank, world),
                                        n_poses=args.n_poses, width=args.width,
                                        height_px=args.height)
    t_gen = time.time() - t0
    ctx = Lodge(local_rank)
    if args.bin_log2 is not None:
        ctx.set_bin_size(args.bin_log2)
    t0 = time.time()
    sid = ctx.load_scene(scene)
    t_load = time.time() - t0
    n_total = scene.n_total
    P = args.poses_per_step
    npix = args.width * args.height
    out = torch.empty(npix * 3, dtype=torch.float32, device=dev)
    # a step's P consecutive poses go to one render call (one image each)
    out_step = torch.empty(P * npix * 3, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def frames(step):
        return [cams[(step * P + j) % len(cams)] for j in range(P)]

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(mode, steps):
        def run():
            for s in range(steps):
                if args.per_frame_calls:
                    for cam in frames(s):
                        ctx.render(sid, mode, cam, out=out)
                else:
                    ctx.render(sid, mode, frames(s), out=out_step)

        def clock(fn):
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / 1e3

        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        return timed_region(run, world, sync=torch.cuda.synchronize, clock=clock, device=dev)

    def frame_latency(mode, n):
        """Device time of single-camera render calls, one frame at a time
        (each call waits for its frame): the latency of one frame."""
        lat = []
        for j in range(n):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.render(sid, mode, cams[j % len(cams)], out=out)
            b.record(stream)
            b.synchronize()
            lat.append(a.elapsed_time(b))
        return lat

    # warm-up, the same calls as the timed steps (grows every scratch buffer,
    # of both slots a step's frames alternate between, to its steady size)
    for s in range(args.warmup):
        if args.per_frame_calls:
            for cam in frames(s):
                ctx.render(sid, CHUNK_BLEND, cam, out=out)
        else:
            ctx.render(sid, CHUNK_BLEND, frames(s), out=out_step)
    ctx.render(sid, FULL, frames(0)[:2], out=out_step)
    torch.cuda.synchronize()

    # ---- timed: LOD + chunk + opacity blending.  No event timing inside the
    # timed region (the counters of frames, keys and launches still run).
    clk = ClockSampler(local_rank)
    ctx.profile_enable(False)
    clk.start()
    # NVTX range "timed_chunk_blend" marks the timed launches for profilers
    # (ncu --nvtx --nvtx-include timed_chunk_blend/)
    torch.cuda.nvtx.range_push("timed_chunk_blend")
    t_blend = timed(CHUNK_BLEND, args.steps)
    torch.cuda.nvtx.range_pop()
    clocks = clk.stop()
    prof_timed = ctx.profile_read()
    n_frames = args.steps * P
    value = job_throughput(n_frames, world, t_blend)

    # ---- full detail on the same poses
    fsteps = args.full_steps if args.full_steps is not None else max(1, args.steps // 2)
    ctx.profile_enable(False)
    torch.cuda.nvtx.range_push("timed_full")
    t_full = timed(FULL, fsteps)
    torch.cuda.nvtx.range_pop()
    prof_full_timed = ctx.profile_read()
    full_fps = job_throughput(fsteps * P, world, t_full)

    # ---- single frames, one call each: the latency of a frame and, with
    # event timing per stage, the stage breakdown and the roofline (frames of
    # one call overlap on two streams, which would blur per-stage events)
    ctx.profile_enable(True)
    n_lat = min(len(cams), 100)
    lat = frame_latency(CHUNK_BLEND, n_lat)
    prof = ctx.profile_read()
    # the same frames again in counting mode (untimed): the compositing's
    # evaluated and composited (pixel, Gaussian) pairs, for its roofline
    ctx.profile_enable(True, count_pairs=True)
    frame_latency(CHUNK_BLEND, n_lat)
    prof_cnt = ctx.profile_read()
    ctx.profile_enable(True)
    lat_full = frame_latency(FULL, 10)
    prof_full = ctx.profile_read()
    ctx.profile_enable(False)

    # ---- the paper's timing protocol (supplementary "Evaluation details"):
    # each pose rendered alone 7 times after 3 warm-up renders, the median
    # kept, FPS = 1 / mean over poses (rendering only, no copy to the host)
    def paper_fps(mode, poses):
        meds = []
        for j in poses:
            cam = cams[j % len(cams)]
            ts = []
            for r in range(10):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.render(sid, mode, cam, out=out)
                b.record(stream)
                b.synchronize()
                if r >= 3:
                    ts.append(a.elapsed_time(b))
            meds.append(float(np.median(ts)))
        return 1e3 / float(np.mean(meds))

    proto_poses = list(range(0, len(cams), max(len(cams) // 30, 1)))[:30]
    paper_protocol = {"chunk_blend_fps": round(paper_fps(CHUNK_BLEND, proto_poses), 1),
                      "full_fps": round(paper_fps(FULL, proto_poses[:10]), 1),
                      "poses": len(proto_poses),
                      "protocol": "each pose rendered alone 7 times after 3 warm-up renders, median kept, "
                                  "FPS = 1 / mean over poses (full detail: the first 10 of the poses)"}

    # ---- end to end through the host-buffer entry point (camera H2D, image D2H)
    host = torch.empty(P * npix * 3, dtype=torch.float32, pin_memory=True).numpy().reshape(-1)
    e2e_steps = args.steps
    # untimed warm-up calls (the first one sizes the device staging)
    for s in range(args.warmup):
        ctx.render_host(sid, CHUNK_BLEND, frames(s), host)
    def run_e2e():
        # one host-buffer call per step: its cameras in, its images out
        for s in range(e2e_steps):
            ctx.render_host(sid, CHUNK_BLEND, frames(args.warmup + s), host)

    t_e2e = timed_region(run_e2e, world, sync=torch.cuda.synchronize, device=dev)
    e2e_fps = job_throughput(e2e_steps * P, world, t_e2e)

    # ---- roofline of the dominant kernel stage
    pk, pk_kind = peaks()
    ms = prof["ms"]
    dom = max(ms, key=lambda k: ms[k])
    launches = sum(prof_timed["launches"].values())
    roof = None
    if dom == "blend":
        # bound by FP32 arithmetic.  Algorithmic unit: about 15 FP32 ops per
        # evaluated (pixel, Gaussian) pair (Eq. 1 alpha, transmittance and
        # colour), the exp2 on the MUFU not counted; peak = SMs x 128 FP32
        # lanes x 2 (FMA) x the maximum SM clock.  The flops this kernel's
        # own formulation needs (9.5 per evaluated pair, the shared dx
        # counted once per two pixels, + 9 per composited pair: T (1 - alpha),
        # T alpha and three colour FMAs) are given beside it.
        sm_mhz = pk.get("sm_max_mhz", 2070.0)
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
        nf = max(prof_cnt["frames"], 1)
        pairs = prof_cnt["blend_pairs"] / nf
        flops = 15.0 * pairs
        flops_own = (9.5 * prof_cnt["blend_pairs"] + 9.0 * prof_cnt["blend_pairs_used"]) / nf
        t_launch = ms["blend"] / max(prof["frames"], 1) / 1e3
        ach = flops / t_launch / 1e12
        tr = measured_traffic("blend", 0)
        roof = {"bound": "alu", "achieved": round(ach, 2), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(ach / peak, 4), "traffic": None if tr is None else round(tr), "kernel": "blend",
                "ops_per_evaluated_pair": 15, "flops_per_launch": round(flops),
                "pairs_per_launch": prof_cnt["blend_pairs"] // nf,
                "composited_pairs_per_launch": prof_cnt["blend_pairs_used"] // nf,
                "own_count": {"flops_per_launch": round(flops_own),
                              "achieved": round(flops_own / t_launch / 1e12, 2),
                              "frac": round(flops_own / t_launch / 1e12 / peak, 4)},
                "avg_launch_ms": round(t_launch * 1e3, 5),
                "peak_source": f"{pk_kind} sm_max_mhz x {n_sm} SMs x 128 FP32 lanes x 2"}
    else:
        by = stage_bytes(dom, prof)
        ach = by / (ms[dom] / 1e3) / 1e9
        peak = pk["hbm_gbs"]
        nl = max(prof["launches"][dom], 1)
        # every bin-sort pass processes all of a frame's bin keys
        per_launch_units = prof["bin_keys"] / max(prof["frames"], 1) if dom == "tile_sort" else 0
        tr = measured_traffic(dom, per_launch_units)
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": None if tr is None else round(tr),
                "kernel": dom, "algorithmic_bytes_per_launch": round(by / nl),
                "avg_launch_ms": round(ms[dom] / nl, 5),
                "peak_source": f"{pk_kind} hbm_gbs (burst copy)"}
    stages = {k: round(v / max(prof["frames"], 1), 4) for k, v in ms.items()}
    stages_full = {k: round(v / max(prof_full["frames"], 1), 4) for k, v in prof_full["ms"].items()}
    stage_gbs = {}
    for k in ("project", "depth_sort", "emit", "tile_sort", "ranges"):
        if ms[k] > 0:
            stage_gbs[k] = round(stage_bytes(k, prof) / (ms[k] / 1e3) / 1e9, 1)

    res = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_blend / args.steps * 1e3, 3), "higher_is_better": True,
        "host_enqueue_ms_per_step": round(prof_timed["host_ms"] / args.steps, 3),
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"outdoor LOD scene {n_total} Gaussians "
                               f"({', '.join(str(l.n) for l in scene.levels)}), 16x16 chunks, "
                               f"{len(cams)}-pose trajectory, {args.width}x{args.height}, "
                               "CHUNK_BLEND (LOD + chunks + opacity blending)",
                   "poses_per_step": P, "scale": args.scale,
                   "l2": "inputs larger than L2 (resident scene), consecutive poses, no flush"},
        "full_detail_fps": round(full_fps, 2),
        "speedup_vs_full": round(value / full_fps, 3),
        "mpix_per_s": round(value * npix / 1e6, 1),
        "frame_latency_ms": {"p50": round(float(np.percentile(lat, 50)), 4),
                             "p99": round(float(np.percentile(lat, 99)), 4),
                             "full_p50": round(float(np.percentile(lat_full, 50)), 4)},
        "paper_protocol": paper_protocol,
        "serve_latency": None,
        "per_frame": {"active": prof_timed["active"] // max(prof_timed["frames"], 1),
                      "visible": prof_timed["visible"] // max(prof_timed["frames"], 1),
                      "keys": prof_timed["keys"] // max(prof_timed["frames"], 1),
                      "bin_keys": prof_timed["bin_keys"] // max(prof_timed["frames"], 1),
                      "full_active": prof_full_timed["active"] // max(prof_full_timed["frames"], 1),
                      "full_visible": prof_full_timed["visible"] // max(prof_full_timed["frames"], 1),
                      "full_keys": prof_full_timed["keys"] // max(prof_full_timed["frames"], 1)},
        "stage_ms_per_frame": stages, "stage_ms_per_frame_full": stages_full,
        "stage_gbs": stage_gbs,
        "e2e": {"value": round(e2e_fps, 2), "unit": UNIT, "h2d_bytes_per_step": 104 * P,
                "d2h_bytes_per_step": 4 * 3 * npix * P},
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "setup_s": {"generate": round(t_gen, 1), "load_scene": round(t_load, 1)},
    }
    if not args.no_next:
        res["next_rows"] = run_next_rows(args, ctx, sid, scene, cams, dev)
    ctx.close()
    del out
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args, scene, cams)
    del scene, cams
    if not args.no_serve:
        torch.cuda.empty_cache()
        res["serve_latency"] = run_serve(args, local_rank)
    if not args.no_large:
        torch.cuda.empty_cache()
        res["large_scene"] = run_large(args, local_rank)
    if not args.no_finetune:
        torch.cuda.empty_cache()
        res["finetune_step"] = run_finetune(args, local_rank)
    return res


def run_next_rows(args, ctx, sid, scene, cams, dev):
    """The method's other steps on the bench's scene (device time of
    synchronous calls, host clock): the greedy depth-threshold search, the
    importance scores and visibility filtering of one chunk, one round of the
    per-level build loop on a chunk cell, and the K-means chunk centres.
    Runs last: the filtering edits one chunk's set."""
    import torch
    from paper_2505_23158_gb300 import api, lod_build, synth
    out = {}
    # f1: greedy threshold search over 10 trajectory views, 19 candidates
    views = cams[::30][:10]
    cand = np.arange(5.0, 100.0, 5.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d, _ = ctx.select_thresholds(sid, views, cand)
    t = time.perf_counter() - t0
    out["threshold_search"] = {"ms": round(t * 1e3, 2), "views": len(views), "candidates": int(cand.size),
                               "levels": scene.num_levels, "chosen_m": [round(float(x), 2) for x in d]}
    # f2: importance of one chunk's own set over 8 views inside it, then filtering
    grid = int(round(math.sqrt(scene.chunk_centers.shape[0])))
    chunk = (grid // 2) * grid + grid // 2
    cv = synth.chunk_views(scene, chunk, 7, 8, args.width, args.height)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    score = ctx.importance(sid, api.CHUNK, cv, chunk=chunk)
    torch.cuda.synchronize()
    t_imp = time.perf_counter() - t0
    sel, _ = ctx.select(sid, api.CHUNK, cv[0])
    n_before = sel["n_active"]
    t0 = time.perf_counter()
    n_after = ctx.filter_chunk(sid, chunk, score, 0.02)
    t_f = time.perf_counter() - t0
    out["importance"] = {"ms_per_view": round(t_imp * 1e3 / len(cv), 3), "views": len(cv),
                         "size": f"{args.width}x{args.height}", "chunk_set_before": int(n_before),
                         "chunk_set_after": int(n_after), "filter_ms": round(t_f * 1e3, 2)}
    # f3: the per-level build loop, level 1 of a 200k-Gaussian chunk cell, 8
    # views at 640x360, 3 rounds of 100 steps (the paper: 1000)
    fs = synth.finetune_scene(seed=args.seed + 5, n=200_000)
    fv = synth.finetune_cameras(fs, seed=args.seed + 5, n=8, width=640, height_px=360)
    base = lod_build.level_params(fs.levels[0], dev)
    targets = [ctx.render_params(*base, c, save=False)[0] for c in fv]
    var = lod_build.filter_variance(0.2, 10.0, fv[0].fy)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g1, hist = lod_build.build_level(ctx, [base], base, [10.0], fv, targets, 0.02, var, [0.0], steps=100,
                                     seed=1)
    torch.cuda.synchronize()
    t_b = time.perf_counter() - t0
    out["lod_build"] = {"s_total": round(t_b, 2), "steps": 300, "ms_per_step_incl_evals": round(t_b * 1e3 / 300, 2),
                        "kept": [h["kept"] for h in hist],
                        "loss": [[round(h["loss_pruned"], 5), round(h["loss_tuned"], 5)] for h in hist],
                        "workload": "level 1 (d_1 = 10 m) of a 200k-Gaussian chunk cell, 8 views at 640x360, "
                                    "3 rounds of 100 steps, loss 0.8 L1 + 0.2 (1 - SSIM)"}
    # f4: K-means chunk centres of the trajectory's camera positions (host, FP64)
    pos = synth.camera_positions(cams)
    t0 = time.perf_counter()
    k = api.num_clusters(pos, 10.0)
    init = synth.kmeans_init(len(pos), k, seed=2)
    _, _, it = api.kmeans_centers(pos, init, max_iter=100)
    out["kmeans"] = {"ms": round((time.perf_counter() - t0) * 1e3, 2), "cameras": len(pos), "clusters": int(k),
                     "iterations": int(it)}
    return out


def run_large(args, local_rank):
    """The large indoor+outdoor scene: 60M level-0 Gaussians over 6 levels,
    32x32 chunks, a batch of 64 cameras at 3840x2160 rendered by one call,
    LOD + chunks + opacity blending against full detail (all 60M level-0
    Gaussians) on the same GPU."""
    import torch
    from paper_2505_23158_gb300 import synth
    from paper_2505_23158_gb300.api import CHUNK_BLEND, FULL, Lodge
    t0 = time.time()
    scene, cams = synth.workload_large(seed=args.seed, n_cams=64, scale=args.large_scale)
    t_gen = time.time() - t0
    dev = torch.device("cuda", local_rank)
    npix = cams[0].width * cams[0].height
    out = torch.empty(len(cams) * npix * 3, dtype=torch.float32, device=dev)
    res = {}
    with Lodge(local_rank) as ctx:
        if args.bin_log2 is not None:
            ctx.set_bin_size(args.bin_log2)
        sid = ctx.load_scene(scene)
        for name, mode in (("chunk_blend", CHUNK_BLEND), ("full", FULL)):
            ctx.render(sid, mode, cams, out=out)          # warm-up, grows scratch
            torch.cuda.synchronize()
            ts = []
            for _ in range(3):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                _, st = ctx.render(sid, mode, cams, out=out)
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b))
            res[name] = {"batch_ms": round(float(np.median(ts)), 2),
                         "frames_per_s": round(len(cams) / (float(np.median(ts)) / 1e3), 1),
                         "keys_per_frame": int(np.mean([s["n_keys"] for s in st])),
                         "visible_per_frame": int(np.mean([s["n_visible"] for s in st]))}
    res["speedup_vs_full"] = round(res["full"]["batch_ms"] / res["chunk_blend"]["batch_ms"], 3)
    res["workload"] = (f"large indoor+outdoor scene {scene.n_total} Gaussians over 6 levels, "
                       f"32x32 chunks, 64 cameras at {cams[0].width}x{cams[0].height} per call, "
                       "median of 3 calls")
    res["setup_s"] = round(t_gen, 1)
    return res


def run_finetune(args, local_rank):
    """One fine-tuning step of one level (2M Gaussians of one chunk cell, 32
    views at 1280x720): forward, L1 against the perturbed scene's images and
    the adjoint for every view, then an Adam update of all five parameter
    groups.  Median device time of args.finetune_steps steps after one
    warm-up step."""
    import torch
    from paper_2505_23158_gb300 import synth
    from paper_2505_23158_gb300.api import Lodge, render_differentiable
    t0 = time.time()
    scene = synth.finetune_scene(seed=args.seed, n=2_000_000)
    target = synth.perturb_scene(scene, seed=args.seed + 1)
    cams = synth.finetune_cameras(scene, seed=args.seed, n=32)
    t_gen = time.time() - t0
    dev = torch.device("cuda", local_rank)
    lv, tl = scene.levels[0], target.levels[0]
    n = lv.n

    def params(l, grad):
        return [torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev).requires_grad_(grad)
                for a in (l.means, l.log_scales, l.quats, l.opacity_logits, l.sh.reshape(n, 48))]

    with Lodge(local_rank) as ctx:
        tps = params(tl, False)
        targets = [ctx.render_params(*tps, cam, save=False)[0].clone() for cam in cams]
        ps = params(lv, True)
        opt = torch.optim.Adam(ps, lr=1e-4)

        def step():
            opt.zero_grad()
            total = torch.zeros((), device=dev)
            for cam, tgt in zip(cams, targets):
                img = render_differentiable(ctx, *ps, cam)
                loss = (img - tgt).abs().mean() / len(cams)
                loss.backward()
                total += loss.detach()
            opt.step()
            return total

        losses = [float(step())]
        ts = []
        for _ in range(max(args.finetune_steps, 1)):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            l = step()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
            losses.append(float(l))
    ms = float(np.median(ts))
    return {"workload": "one level of 2M Gaussians (one 62.5 m chunk cell), 32 views at 1280x720, "
                        "L1 against the scene with means + N(0, 0.05 m) and logits + N(0, 0.3); "
                        "a step = forward + adjoint of every view + Adam on all five groups",
            "ms_per_step": round(ms, 2), "views_per_s": round(32 / (ms / 1e3), 1),
            "loss_per_step": [round(x, 6) for x in losses], "setup_s": round(t_gen, 1)}


def cpu_baseline(args, scene, cams, budget_s=None, max_frames=None):
    """The oracle timed on this host's cores on a bounded sample: whole
    CHUNK_BLEND frames of the same trajectory (poses 0, 75, 150, 225, 299
    first, then every 37th) until the time budget is spent (at least one);
    beside it, one full-detail frame at pose 0 and the 4,096-Gaussian plain
    scene at 256x256."""
    import oracle as O
    from paper_2505_23158_gb300 import synth
    budget_s = args.cpu_budget_s if budget_s is None else budget_s
    osc = O.OracleScene(scene)
    ncores = os.cpu_count()
    n = len(cams)
    order = [p for p in (0, 75, 150, 225, 299) if p < n]
    done, spent, idx = 0, 0.0, 0
    while (done == 0 or spent < budget_s) and (max_frames is None or done < max_frames):
        cam = cams[order[idx]] if idx < len(order) else cams[(idx * 37) % n]
        # per-chunk sets are a load-time precompute on both sides; warm them
        A, B, _, _ = O.chunk_pick(osc.centers, cam.center)
        O.chunk_select(osc, A)
        if B >= 0:
            O.chunk_select(osc, B)
        t0 = time.perf_counter()
        g, m, _ = O.active_set(osc, O.MODE_CHUNK_BLEND, cam)
        O.render(osc, cam, g, m, bounds=False)
        spent += time.perf_counter() - t0
        done += 1
        idx += 1
    out = {"value": round(done / spent, 4), "unit": UNIT, "cores": ncores, "kind": "oracle",
           "sample": f"{done} whole CHUNK_BLEND {args.width}x{args.height} frames of the trajectory "
                     f"(poses 0, 75, 150, 225, 299, then every 37th; FP64 binned oracle, OpenMP over "
                     f"tiles), chunk sets precomputed"}
    if max_frames is None:
        t0 = time.perf_counter()
        g, _, _ = O.active_set(osc, O.MODE_FULL, cams[0])
        O.render(osc, cams[0], g, None, bounds=False)
        t_full = time.perf_counter() - t0
        pscene, pcams = synth.workload_plain(0)
        posc = O.OracleScene(pscene)
        t0 = time.perf_counter()
        reps = 0
        while reps < 3 or time.perf_counter() - t0 < 1.0:
            O.render(posc, pcams[0], np.arange(posc.n_total), bounds=False)
            reps += 1
        t_plain = (time.perf_counter() - t0) / reps
        out["full_detail_frames_per_s"] = round(1.0 / t_full, 4)
        out["full_detail_sample"] = f"pose 0 at full detail ({g.size} level-0 Gaussians), {args.width}x{args.height}"
        out["plain_256_frames_per_s"] = round(1.0 / t_plain, 2)
    return out


SERVE_LEVEL0 = (2_000_000, 8_000_000, 16_000_000, 30_000_000)
SERVE_RES = ((640, 360), (1280, 720), (1920, 1080), (3840, 2160))


def serve_requests(rng, scenes, sids, n, rate, t0=0.0):
    """Poisson arrivals at `rate`, uniform scene, street-height pose in the
    inner 80% of the scene (uniform yaw, 10 degree down pitch), resolution
    uniform over SERVE_RES."""
    from paper_2505_23158_gb300 import synth
    from paper_2505_23158_gb300.api import CHUNK_BLEND
    t = t0 + np.cumsum(rng.exponential(1.0 / rate, size=n))
    which = rng.integers(0, len(scenes), size=n)
    res = rng.integers(0, len(SERVE_RES), size=n)
    seeds = rng.integers(0, 2 ** 31, size=n)
    reqs = []
    for i in range(n):
        w, h = SERVE_RES[res[i]]
        cam = synth.random_street_cameras(scenes[which[i]], int(seeds[i]), 1, w, h)[0]
        reqs.append((sids[which[i]], CHUNK_BLEND, cam, float(t[i])))
    return reqs


def serve_summary(reqs, results, rate, duration):
    """Latency percentiles of one serving run, split into queueing (arrival
    to admission), service (admission to image done) and by whether the
    request had to gather a chunk block into HBM."""
    ok = [(q, r) for q, r in zip(reqs, results) if r["status"] == 0]
    lat = np.array([r["latency_s"] for _, r in ok]) * 1e3
    queue = np.array([r["start_s"] - q[3] for q, r in ok]) * 1e3
    serv = np.array([r["finish_s"] - r["start_s"] for _, r in ok]) * 1e3
    up = np.array([r["uploads"] > 0 for _, r in ok], bool)
    t_end = max(r["finish_s"] for r in results) if results else 1.0

    def pct(a, p):
        return round(float(np.percentile(a, p)), 3) if a.size else None

    by_res = {}
    for q, r in ok:
        by_res.setdefault(f"{q[2].width}x{q[2].height}", []).append(r["latency_s"] * 1e3)
    steps = [r["step_frames"] for _, r in ok]
    return {"rate_rps": rate, "duration_s": duration, "requests": len(reqs), "completed": len(ok),
            "throughput_rps": round(len(ok) / t_end, 2),
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
            "queue_p50_ms": pct(queue, 50), "queue_p99_ms": pct(queue, 99),
            "service_p50_ms": pct(serv, 50), "service_p99_ms": pct(serv, 99),
            "p99_ms_with_upload": pct(lat[up], 99), "p99_ms_no_upload": pct(lat[~up], 99),
            "requests_with_upload": int(up.sum()),
            # per request: the frames of the step that served it (request-weighted)
            "mean_frames_per_step": round(float(np.mean(steps)), 2) if steps else None,
            "p99_ms_by_resolution": {k: round(float(np.percentile(v, 99)), 3) for k, v in sorted(by_res.items())}}


def run_serve(args, local_rank):
    """Serving stream over four streamed scenes under an HBM budget: request
    steps (the requests that have arrived, composited by one persistent
    launch per step) at the configuration's rate and at higher rates, and
    the same stream on slot workers."""
    from paper_2505_23158_gb300 import synth
    from paper_2505_23158_gb300.api import STREAMED, Lodge
    t0 = time.time()
    scenes = []
    for i, n0 in enumerate(SERVE_LEVEL0):
        n = int(n0 * args.serve_scale)
        side = math.sqrt(n / 16.0)          # constant density: 16 level-0 Gaussians per m^2
        scenes.append(synth.outdoor_scene(seed=args.seed + 10 + i, n0=n, num_levels=4, extent=side,
                                          grid=16))
    t_gen = time.time() - t0
    budget = int(args.serve_budget_gb * (1 << 30))
    rates = [(args.serve_rate, args.serve_seconds)] + [(r, d) for r, d in ((1000.0, 10.0), (4000.0, 5.0))
                                                         if r > args.serve_rate]
    with Lodge(local_rank, hbm_budget_bytes=budget) as ctx:
        if args.bin_log2 is not None:
            ctx.set_bin_size(args.bin_log2)
        t0 = time.time()
        sids = [ctx.load_scene(sc, STREAMED) for sc in scenes]
        t_load = time.time() - t0
        rng = np.random.default_rng(args.seed + 77)
        warm = serve_requests(rng, scenes, sids, int(args.serve_warmup_s * args.serve_rate), args.serve_rate)
        ctx.serve(warm, realtime=True, batch=args.serve_batch)
        r0 = ctx.residency_stats()
        clk = ClockSampler(local_rank)
        clk.start()
        sweep = []
        for rate, dur in rates:
            reqs = serve_requests(rng, scenes, sids, int(dur * rate), rate)
            res, _ = ctx.serve(reqs, realtime=True, batch=args.serve_batch)
            sweep.append(serve_summary(reqs, res, rate, dur))
        clocks = clk.stop()
        r1 = ctx.residency_stats()
        # the configuration's rate on slot workers (one request per slot,
        # each composited by its own launch)
        sreqs = serve_requests(rng, scenes, sids, int(args.serve_slot_seconds * args.serve_rate),
                               args.serve_rate)
        sres, _ = ctx.serve(sreqs, slots=args.serve_slots, realtime=True)
        slots = serve_summary(sreqs, sres, args.serve_rate, args.serve_slot_seconds)
        slots["slots"] = args.serve_slots
    main = sweep[0]
    uploads = r1["block_uploads"] - r0["block_uploads"]
    hits = r1["block_hits"] - r0["block_hits"]
    return {
        **main, "batch": args.serve_batch, "sweep": sweep[1:], "slot_workers": slots,
        "hbm_budget_gb": args.serve_budget_gb,
        "scenes_level0": [int(n * args.serve_scale) for n in SERVE_LEVEL0],
        "residency": {"block_uploads": uploads, "block_hits": hits,
                      "hit_rate": round(hits / max(hits + uploads, 1), 3),
                      "evictions": r1["block_evictions"] - r0["block_evictions"],
                      "upload_gb": round((r1["upload_bytes"] - r0["upload_bytes"]) / 1e9, 2),
                      "hbm_used_gb": round(r1["hbm_used"] / (1 << 30), 2)},
        "clocks": clocks, "setup_s": {"generate": round(t_gen, 1), "load": round(t_load, 1)},
        "workload": "4 streamed outdoor LOD scenes (4 levels, constant density, 16x16 chunks), "
                    "Poisson arrivals, uniform scene, random street-height pose, resolution "
                    f"uniform over 640x360/1280x720/1920x1080/3840x2160, CHUNK_BLEND; steps of at most "
                    f"{args.serve_batch} arrived requests, {args.serve_warmup_s:g} s warm-up",
    }


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from paper_2505_23158_gb300 import synth
    import oracle as O
    scene, cams = synth.workload_outdoor(seed=args.seed, n_poses=args.n_poses, scale=args.scale,
                                         width=args.width, height_px=args.height)
    osc = O.OracleScene(scene)

    def step(s):
        cam = cams[(s * 37) % len(cams)]
        A, B, _, _ = O.chunk_pick(osc.centers, cam.center)
        O.chunk_select(osc, A)
        if B >= 0:
            O.chunk_select(osc, B)
        t0 = time.perf_counter()
        g, m, _ = O.active_set(osc, O.MODE_CHUNK_BLEND, cam)
        O.render(osc, cam, g, m, bounds=False)
        return time.perf_counter() - t0

    for s in range(args.warmup):
        step(s)
    ts = [step(args.warmup + s) for s in range(args.steps)]
    t = sum(ts)
    value = args.steps / t
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t / args.steps * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"outdoor LOD scene {scene.n_total} Gaussians, 16x16 chunks, "
                                   f"{args.width}x{args.height}, CHUNK_BLEND; one whole frame per step",
                       "scale": args.scale},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": "one whole CHUNK_BLEND frame per step (FP64 binned oracle, "
                                       "OpenMP over tiles), chunk sets precomputed"},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res = run_lodge(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
