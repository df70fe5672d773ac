"""Autotuner of the batched encoder iteration.

The tunable is the launch schedule of a batch: per kernel class (entropy model, synthesis,
residual convs, the rest) the fraction of each job's single-image CTA count used when all jobs run
in one launch.  Fewer CTAs per job mean fewer partial gradients to reduce and less tail; more CTAs
mean more parallelism per image.  The best point depends on the mix of image sizes, so it is
measured: every candidate runs one graph-captured iteration on clones of the jobs' states (the real
states are not advanced) and is timed with CUDA events.  Results are cached per device and size mix.
"""
from __future__ import annotations

import json
import os

import torch

from . import lib as cc

CANDIDATES = [
    (1.0, 1.0, 1.0, 1.0),
    (0.5, 0.5, 0.5, 1.0),
    (0.5, 1.0, 1.0, 0.5),
    (0.25, 0.5, 0.5, 0.5),
    (0.25, 0.25, 0.25, 0.25),
    (0.125, 0.25, 0.25, 0.25),
]

_cache: dict = {}


def _key(shapes, device):
    name = torch.cuda.get_device_name(device)
    return f"{name}|" + ",".join(f"{h}x{w}" for h, w in sorted(shapes))


def _clone_jobs(jobs):
    return [(img, st.clone(), hp) for img, st, hp in jobs]


def time_schedule(jobs, schedule, repeats=5, warmup=2):
    """Milliseconds per batched iteration (graph replay, events), on cloned states."""
    be = cc.BatchEncoder(_clone_jobs(jobs), schedule=schedule, rd_capacity=1)
    try:
        g = be.graph(1)
        for _ in range(warmup):
            g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(repeats):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / repeats
    finally:
        be.close()


def tune(jobs, candidates=CANDIDATES, repeats=5, cache_file=None):
    """Returns (best Schedule, {candidate: ms}).  Cached per device and size mix."""
    shapes = [(int(img.shape[1]), int(img.shape[2])) for img, _, _ in jobs]
    device = jobs[0][0].device
    key = _key(shapes, device)
    if cache_file and not _cache and os.path.exists(cache_file):
        with open(cache_file) as f:
            _cache.update({k: tuple(v) for k, v in json.load(f).items()})
    if key in _cache:
        return cc.Schedule(*_cache[key]), {}
    timings = {}
    for cand in candidates:
        timings[cand] = time_schedule(jobs, cc.Schedule(*cand), repeats=repeats)
    best = min(timings, key=timings.get)
    _cache[key] = best
    if cache_file:
        os.makedirs(os.path.dirname(os.path.abspath(cache_file)), exist_ok=True)
        with open(cache_file, "w") as f:
            json.dump({k: list(v) for k, v in _cache.items()}, f)
    return cc.Schedule(*best), timings
