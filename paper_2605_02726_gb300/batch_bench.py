"""Mixed-size batch benchmark: 32 images with sizes drawn uniformly from {256x256, 512x768,
768x512, 1024x1024, 1536x1024}, each with its own decoder and Adam state.

Compares the plain path (one image at a time, its iterations launched kernel by kernel, no graph)
with the batched path (all images advance together: one launch per kernel, the iteration captured
in a CUDA graph, the launch schedule picked by the autotuner).  Both start from the same states,
and the final rate-distortion losses are reported side by side: with the default schedule they are
bitwise equal (the GPU tests check this); a tuned schedule changes the number of per-CTA partial
gradients, hence their summation order, and after hundreds of iterations the two trajectories
differ by a few percent in loss, as any two summation orders do.

  python -m paper_2605_02726_gb300.batch_bench [--images 32] [--iters 2000]
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import autotune, inputs
from . import lib as cc


def make_jobs(n_images, seed0=inputs.SEED0, lam=1e-3):
    jobs = []
    for j, (H, W) in enumerate(inputs.batch_workload(n_images, seed0)):
        img = torch.tensor(inputs.image(H, W, seed=seed0 + j), device="cuda")
        lat, par = inputs.initial_state(H, W, seed=seed0 + 100 + j)
        st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"))
        jobs.append((img, st, cc.hparams(lam=lam, seed=seed0 + j)))
    return jobs


def plain(jobs, iters):
    """One image per launch sequence, no graph; returns (seconds, final losses)."""
    out = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for img, st, hp in jobs:
        H, W = img.shape[1], img.shape[2]
        rd = torch.zeros(iters, 3, dtype=torch.float64, device="cuda")
        cc.encode_step(img, st, iters, H=H, W=W, hp=hp, ws=cc.workspace(H, W), rd=rd)
        out.append(rd[-1, 0])
    torch.cuda.synchronize()
    return time.perf_counter() - t0, torch.stack(out).cpu().numpy()


def plain_by_size(jobs, iters):
    """Plain-path rate of each distinct image size alone (Mpixel-iterations/s): how far one image
    of that size fills the GPU by itself, the ceiling that batching works against."""
    rates = {}
    for img, st, hp in jobs:
        H, W = img.shape[1], img.shape[2]
        key = f"{H}x{W}"
        if key in rates:
            continue
        s = st.clone()
        ws = cc.workspace(H, W)
        rd = torch.zeros(iters, 3, dtype=torch.float64, device="cuda")
        cc.encode_step(img, s, 5, H=H, W=W, hp=hp, ws=ws, rd=rd)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cc.encode_step(img, s, iters, H=H, W=W, hp=hp, ws=ws, rd=rd)
        torch.cuda.synchronize()
        rates[key] = H * W * iters / (time.perf_counter() - t0) / 1e6
    return rates


def batched(jobs, iters, schedule, graph_iters=10):
    be = cc.BatchEncoder(jobs, schedule=schedule, rd_capacity=graph_iters)
    g = be.graph(graph_iters)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = 0
    while done + graph_iters <= iters:
        g.replay()
        done += graph_iters
    if done < iters:
        be.step(iters - done)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    last = (iters - done - 1) if done < iters else graph_iters - 1
    losses = be.records()[last, :, 0].cpu().numpy()
    be.close()
    return dt, losses


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--images", type=int, default=32)
    ap.add_argument("--iters", type=int, default=2000)
    a = ap.parse_args()
    jobs = make_jobs(a.images)
    pix = sum(img.shape[1] * img.shape[2] for img, _, _ in jobs)
    sched, timings = autotune.tune(jobs, repeats=3)
    plain_jobs = [(img, st.clone(), hp) for img, st, hp in jobs]
    t_plain, l_plain = plain(plain_jobs, a.iters)
    batch_jobs = [(img, st.clone(), hp) for img, st, hp in jobs]
    t_batch, l_batch = batched(batch_jobs, a.iters, sched)
    rel = float(np.max(np.abs(l_batch - l_plain) / np.abs(l_plain)))
    by_size = plain_by_size(jobs, min(a.iters, 500))
    print(json.dumps({
        "workload": f"{a.images} images {sorted(set(tuple(img.shape[1:]) for img, _, _ in jobs))}, {a.iters} iterations",
        "megapixels": pix / 1e6,
        "plain_mpix_iter_per_s": pix * a.iters / t_plain / 1e6,
        "batched_mpix_iter_per_s": pix * a.iters / t_batch / 1e6,
        "speedup": t_plain / t_batch,
        "plain_alone_mpix_iter_per_s": by_size,
        "schedule": list(sched.as_tuple()),
        "autotune_ms": {",".join(map(str, k)): v for k, v in timings.items()},
        "final_loss_max_rel_diff": rel,
    }), flush=True)


if __name__ == "__main__":
    main()
