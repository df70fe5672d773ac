#!/usr/bin/env python
"""Encoder-step benchmark: Mpixel-iterations/s of the fused forward + backward + Adam iteration.

Workload: one 512x768 RGB image from the seeded 1/f^2 generator with sigma 0.02 texture noise,
the L=7 architecture, lambda 1e-3, Adam lr 1e-2 (a stand-in for a Kodak-sized image; no
dataset is available).  A step is one encoder iteration over the whole image.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one independent replica per GPU (launched with torch.distributed.run), no
collective on the data path; the value is the whole-job rate (sum of the replicas' work over the
slowest replica's time).  --impl reference times the FP64 CPU oracle on the host cores instead.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H, W = 512, 768
LAM = 1e-3
SEED = 20260
METRIC = "encoder Mpixel-iterations/s (fwd+bwd+Adam)"
UNIT = "Mpixel-iter/s"
WORKLOAD = "512x768 RGB 1/f^2 + texture noise, L=7 Cool-chic decoder (ARM 16x2 + IFCE, 8-tap upsampler, syn 7-40-3 + 2 res 3x3), lambda 1e-3"

# Algorithmic work of the entropy-model kernel (forward + adjoint + parameter gradients) per
# latent: 3 x 648 MAC of the ARM matrices (forward, input adjoint, weight gradient) plus the IFCE
# matrices of grids 0..2 (3 x 4 x nin MAC), 2 FLOP per MAC.
ARM_MAC_PER_LATENT = 3 * 648
IFCE_NIN = (6, 5, 4)
# Unit-count figure of the FP32 pipe (152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz), reported beside
# the peak measured in the same run (coolchic_measure_peak), which is the roofline denominator.
FP32_UNIT_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# DRAM bytes (read + write) per launch of the entropy-model kernel, from the full ncu capture of
# the current kernel at 512 x 768 (cold caches: 2.17 MB read, 0.41 MB written; the 33.5 MB of
# context-gradient planes it writes are still in L2 when the launch ends).
ARM_TRAFFIC_BYTES = 2.58e6
# Algorithmic work of one whole encoder iteration per pixel: 1522 forward MAC per pixel (ARM 864,
# IFCE 30, upsampling 45, synthesis 1x1 421, 3x3 convs 162), the adjoint and the parameter
# gradients twice that again, 2 FLOP per MAC.
STEP_FLOP_PER_PIXEL = 3 * 1522 * 2

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def grid_sizes(h, w):
    return [(-(-h // (1 << k)), -(-w // (1 << k))) for k in range(7)]


def arm_flops(h, w):
    g = grid_sizes(h, w)
    n = sum(a * b for a, b in g)
    mac = ARM_MAC_PER_LATENT * n + sum(3 * 4 * IFCE_NIN[k] * g[k][0] * g[k][1] for k in range(3))
    return 2.0 * mac


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cores_used():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else os.cpu_count()


def oracle_rate(h, w, iters, seed):
    """Oracle pixel-iterations/s over `iters` iterations of an h x w image (as it stands)."""
    import oracle
    from paper_2605_02726_gb300 import inputs
    img = inputs.image(h, w, seed=seed, texture_sigma=0.02)
    lat, par = inputs.initial_state(h, w, seed=seed + 1)
    st = oracle.State(lat, par)
    t0 = time.perf_counter()
    oracle.encode(img, st, iters, lam=LAM, seed=seed)
    dt = time.perf_counter() - t0
    return h * w * iters / dt / 1e6, dt


def max_over_ranks(x: float, world: int, device) -> float:
    """Every rank's x reduced by max (the job ends with its slowest rank); x as is for one rank.
    device: where the process group's backend takes tensors (cuda for nccl, cpu for gloo)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, ms: float) -> float:
    """Whole-job throughput in millions of units per second: the units of all ranks over the
    slowest rank's time (every rank runs the same work)."""
    return world * units_per_rank / (ms * 1e-3) / 1e6


def run_reference(args, rank):
    """The FP64 oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    budget = 150.0 / (args.steps + args.warmup)  # seconds per step
    rate0, _ = oracle_rate(32, W, 1, SEED)        # calibration on a 32-row band
    rows = int(min(H, max(8, budget * rate0 * 1e6 / W)))
    for _ in range(args.warmup):
        oracle_rate(rows, W, 1, SEED)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_rate(rows, W, 1, SEED)
        times.append(dt)
    tot = sum(times)
    value = rows * W * args.steps / tot / 1e6
    sample = f"one encoder iteration per step on a {rows}x{W} band of the 512x768 workload"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_rows": rows},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores_used(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-iters", type=int, default=10, help="oracle iterations of the CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--min-seconds", type=float, default=2.0,
                    help="repeat the K timed steps (whole passes) until the timed region lasts this long")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2605_02726_gb300 import inputs, lib as cc

    dev = torch.device("cuda", local)
    img_np = inputs.image(H, W, seed=SEED + 97 * rank, texture_sigma=0.02)
    lat, par = inputs.initial_state(H, W, seed=SEED + 97 * rank + 1)
    image = torch.tensor(img_np, device=dev)
    st = cc.EncoderState(torch.tensor(lat, device=dev), torch.tensor(par, device=dev))
    ws = cc.workspace(H, W, device=dev)
    hp = cc.hparams(lam=LAM, seed=SEED + rank)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        cc.encode_step(image, st, 1, H=H, W=W, hp=hp, ws=ws)
    barrier()

    # pipe ceilings of this GPU, measured now (FP32 FMA and TF32 mma.sync), before the timed region
    fp32_peak, _ = cc.measure_peak(cc.PEAK_FP32_FMA)
    tf32_peak, _ = cc.measure_peak(cc.PEAK_TF32_MMA)
    for _ in range(3):
        cc.encode_step(image, st, 1, H=H, W=W, hp=hp, ws=ws)
    barrier()

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    # the entropy-model kernel is timed by event pairs around its launch in the first tenth of the
    # first pass's steps (those steps launch eagerly; the rest replay the library's CUDA graph of
    # the call)
    K_arm = max(3, K // 10)
    cc.timing_enable(cc.KERNEL_ARM, K_arm)

    def timed_pass():
        """Exactly K steps between a barrier + synchronize on both sides; their summed event time."""
        barrier()
        for i in range(K):
            flush.zero_()  # L2 flushed between timed iterations (outside the events)
            ev[i][0].record(stream)
            cc.encode_step(image, st, 1, H=H, W=W, hp=hp, ws=ws)
            ev[i][1].record(stream)
        barrier()
        return sum(a.elapsed_time(b) for a, b in ev)

    # The K timed steps are repeated in whole passes until the timed region lasts --min-seconds,
    # so that the clock sampler sees the GPU under load; every rank runs the same number of passes.
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        tot_ms = timed_pass()
        first_s = time.perf_counter() - t_wall
        passes = max(1, int(np.ceil(args.min_seconds / max(first_s, 1e-6))))
        passes = int(max_over_ranks(passes, world, dev))
        for _ in range(passes - 1):
            tot_ms += timed_pass()
        t_wall = time.perf_counter() - t_wall
    arm_ms, arm_n = cc.timing_collect()
    cc.timing_disable()
    tot_ms = max_over_ranks(tot_ms, world, dev)
    ms_per_step = tot_ms / (K * passes)
    value = job_rate(world, H * W * K * passes, tot_ms)

    # end to end through the host-buffer entry point (coolchic_encode_step_host): every step copies
    # the image from pinned host memory into the workspace, runs the iteration and copies its loss
    # record back to pinned host memory, all inside the events
    host_img = torch.tensor(img_np).pin_memory()
    host_rd = torch.zeros(3, dtype=torch.float64).pin_memory()
    ws_io = cc.workspace(H, W, device=dev, host_io=True)
    Ke = min(K, 200)
    eve = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(Ke)]
    for _ in range(3):
        cc.encode_step_host(host_img, st, 1, H=H, W=W, hp=hp, ws=ws_io, rd_host=host_rd)
    barrier()
    for i in range(Ke):
        flush.zero_()
        eve[i][0].record(stream)
        cc.encode_step_host(host_img, st, 1, H=H, W=W, hp=hp, ws=ws_io, rd_host=host_rd)
        eve[i][1].record(stream)
    barrier()
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in eve) / Ke, world, dev)
    loss_now = float(host_rd[0])

    clocks = clk.summary()
    if clocks.get("sm_mhz"):
        clocks["ms_per_step_x_sm_mhz"] = ms_per_step * clocks["sm_mhz"]
    arm_avg_s = arm_ms * 1e-3 / max(arm_n, 1)
    achieved = arm_flops(H, W) / arm_avg_s / 1e12
    step_achieved = value * 1e6 * STEP_FLOP_PER_PIXEL / 1e12
    roofline = {"kernel": "k_arm (entropy model fwd+adjoint)", "bound": "alu", "achieved": achieved,
                "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                "traffic": ARM_TRAFFIC_BYTES, "launch_ms": arm_avg_s * 1e3,
                "share_of_step": (arm_ms / max(arm_n, 1)) / ms_per_step,
                "peak_source": "measured in this run: FP32 FMA pipe (coolchic_measure_peak), "
                               f"unit-count figure {FP32_UNIT_TFLOPS:.1f}",
                "tensor_pipe": {"peak": tf32_peak, "peak_source": "measured in this run: mma.sync.m16n8k8 TF32",
                                "frac_algorithmic": achieved / tf32_peak,
                                "frac_executed_hi_lo": 3.0 * achieved / tf32_peak},
                "step": {"flop_per_pixel": STEP_FLOP_PER_PIXEL, "achieved": step_achieved,
                         "frac": step_achieved / fp32_peak}}

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            v, dt = oracle_rate(H, W, args.cpu_iters, SEED)
            cpu = {"value": v, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
                   "sample": f"{args.cpu_iters} encoder iterations of the 512x768 workload ({dt:.1f} s)"}
        launches_per_step = cc.kernel_launches(H, W, 1)  # one encode_step call of one iteration per step
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "passes": passes, "timed_steps": K * passes,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "image": [H, W], "latents": cc.latent_count(H, W),
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "flushed between timed iterations (256 MB write outside the events)",
                       "launch": f"{launches_per_step} kernels per iteration, replayed from the library's CUDA "
                                 f"graph of the call (the first {K_arm} timed steps eager, the entropy model timed)",
                       "timing": f"{passes} passes of the {K} timed steps (each between barriers), "
                                 f"repeated until the timed region lasted {args.min_seconds} s"},
            "e2e": {"value": job_rate(world, H * W, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": int(host_img.numel() * 4), "d2h_bytes_per_step": 24,
                    "ms_per_step": e2e_ms, "loss_readback": loss_now,
                    "call": "coolchic_encode_step_host (host image in, host loss record out)"},
            "gpu_launches": launches_per_step * K * passes,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "wall_s": t_wall,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
