"""Continuous-batching encode server.

Encode requests (an image, lambda, a seed, an iteration budget) arrive over time.  A request is
admitted, first come first served, when a slot is free (at most `slots` jobs still have iterations
to run; 0 = no limit) and its device memory (image, latents, parameters, Adam state, workspace) fits
in the HBM budget next to the jobs already resident; admitted jobs stay resident on the device and advance
together: every tick runs up to `tick_iters` encoder iterations of all active jobs through the
batched launches (one launch per kernel for the whole set).  A job leaves when it has done its
iterations (its final state and last loss record are copied to the host) or is cancelled; its
memory is released and queued requests are admitted.  Each job's trajectory is the one it would
have alone: jobs never share state, and a job's kernels see only its own buffers.

Ticks are pipelined: `run` keeps up to two ticks queued on the GPU stream.  While tick t runs, the
host retires tick t-1 (copies the finished jobs' results on a side stream ordered after that tick
alone, releases their memory), admits new arrivals and plans tick t+1; a job's iteration count is
known in advance, so the jobs that finish with tick t are left out of tick t+1 before t completes.
A membership change builds the next plan with the non-blocking coolchic_batch_create_async (the
plan is copied on the stream from a pinned buffer), so the GPU never waits for the host between
ticks.  The latency of a request runs from its arrival to the host's retirement of its last tick.

Slots: a few jobs of a megapixel or more already keep the GPU busy, so admitting every request that
fits in memory only makes all of them share the GPU and finish together, late; a few slots let the
jobs at the head of the queue finish first at about the same throughput.

`python -m paper_2605_02726_gb300.serve` runs the Poisson-arrival benchmark (sizes 512x768,
1024x1024, 2048x1365, 2048x2048 weighted .4/.3/.2/.1; lambda in {1e-4, 1e-3, 1e-2}; 80 GB budget;
`--requests` per offered rate, `--slots`) and prints one JSON line per rate with p50/p99 latency,
the offered and the served request rates and pixel-iterations per second.
"""
from __future__ import annotations

import argparse
import collections
import ctypes
import json
import math
import time

import numpy as np
import torch

from . import inputs
from . import lib as cc


def job_bytes(H: int, W: int) -> int:
    """Device bytes a resident job holds: image, state (latents, params, Adam moments, step),
    and its workspace."""
    n = cc.latent_count(H, W)
    ws = int(cc._lib.coolchic_workspace_bytes(ctypes.byref(cc.arch(H, W)), 0))
    return 4 * 3 * H * W + 4 * 3 * n + 4 * 3 * cc.N_PARAMS + 8 + ws + 512


Request = collections.namedtuple("Request", "rid arrival H W lam seed iters image")
Tick = collections.namedtuple("Tick", "event batch jobs n finishing")


class Job:
    def __init__(self, req: Request, device):
        self.req = req
        self.image = req.image.to(device, non_blocking=True) if req.image.device.type != "cuda" else req.image
        lat, par = inputs.initial_state(req.H, req.W, seed=req.seed + 1)
        self.state = cc.EncoderState(torch.tensor(lat, device=device), torch.tensor(par, device=device))
        self.hp = cc.hparams(lam=req.lam, seed=req.seed)
        self.ws = cc.workspace(req.H, req.W, device=device)
        self.done_iters = 0     # iterations retired
        self.planned = 0        # iterations queued on the GPU
        self.bytes = job_bytes(req.H, req.W)
        self.admitted = None
        self.finished = None
        self.last_rd = None
        self.final = None
        self.cancelled = False


class EncodeServer:
    def __init__(self, hbm_budget: int, tick_iters: int = 50, schedule=None, device="cuda", max_inflight: int = 2,
                 slots: int = 0):
        self.budget = int(hbm_budget)
        self.slots = max(0, int(slots))  # jobs with iterations left at most (0: memory alone decides)
        self.tick_iters = int(tick_iters)
        self.schedule = schedule
        self.device = torch.device(device)
        self.stream = torch.cuda.current_stream(self.device)
        self.copy_stream = torch.cuda.Stream(self.device)
        self.max_inflight = max(1, int(max_inflight))
        self.queue: collections.deque = collections.deque()
        self.active: list[Job] = []
        self.done: dict[int, Job] = {}
        self.failed: dict[int, str] = {}
        self.inflight: collections.deque = collections.deque()
        self.in_use = 0
        self.peak_in_use = 0
        self.batch = None
        self.batch_key = None
        self.ticks = 0
        self.plans = 0
        self._next = 0

    # -- request intake -----------------------------------------------------------------------
    def submit(self, image, lam: float, seed: int, iters: int, arrival: float | None = None) -> int:
        """Queue a request; malformed ones are rejected at once (recorded in `failed`)."""
        rid = self._next
        self._next += 1
        arrival = time.perf_counter() if arrival is None else arrival
        img = torch.as_tensor(image)
        if img.dim() != 3 or img.shape[0] != 3 or not (1 <= img.shape[1] <= 16384 and 1 <= img.shape[2] <= 16384):
            self.failed[rid] = "malformed image shape"
            return rid
        if not (math.isfinite(lam) and lam >= 0.0) or iters < 1:
            self.failed[rid] = "invalid lambda or iteration count"
            return rid
        H, W = int(img.shape[1]), int(img.shape[2])
        if job_bytes(H, W) > self.budget:
            self.failed[rid] = "larger than the whole HBM budget"
            return rid
        self.queue.append(Request(rid, arrival, H, W, float(lam), int(seed), int(iters), img.float().contiguous()))
        return rid

    def cancel(self, rid: int) -> bool:
        """Cancel a queued or resident request; a resident one leaves at its next tick boundary
        (its memory is released once the ticks already queued have retired)."""
        for q in list(self.queue):
            if q.rid == rid:
                self.queue.remove(q)
                self.failed[rid] = "cancelled"
                return True
        for j in self.active:
            if j.req.rid == rid and not j.cancelled:
                j.cancelled = True
                self.failed[rid] = "cancelled"
                if not any(j in t.jobs for t in self.inflight):
                    self._release(j)
                return True
        return False

    # -- scheduling ---------------------------------------------------------------------------
    def _release(self, job: Job):
        if job in self.active:
            self.active.remove(job)
            self.in_use -= job.bytes

    def _running(self) -> int:
        # jobs that still have iterations to queue (a job whose last tick is queued frees its slot)
        return sum(1 for j in self.active if j.planned < j.req.iters and not j.cancelled)

    def _admit(self, now: float):
        while self.queue and self.queue[0].arrival <= now:
            if self.slots and self._running() >= self.slots:
                break  # FIFO: wait for a slot
            need = job_bytes(self.queue[0].H, self.queue[0].W)
            if self.in_use + need > self.budget:
                break  # FIFO: wait for memory
            req = self.queue.popleft()
            job = Job(req, self.device)
            job.admitted = now
            self.active.append(job)
            self.in_use += job.bytes
            self.peak_in_use = max(self.peak_in_use, self.in_use)

    def _plan(self, jobs):
        key = tuple(j.req.rid for j in jobs)
        if key != self.batch_key:
            # the previous plan stays alive in the ticks that use it; a new one is uploaded on the
            # stream without blocking
            self.batch = cc.BatchEncoder([(j.image, j.state, j.hp) for j in jobs], schedule=self.schedule,
                                         rd_capacity=self.tick_iters, workspaces=[j.ws for j in jobs],
                                         stream=self.stream)
            self.batch_key = key
            self.plans += 1
        return self.batch

    def _launch(self) -> int:
        """Queue one tick of the jobs that still have iterations; returns its iteration count."""
        jobs = [j for j in self.active if j.planned < j.req.iters and not j.cancelled]
        if not jobs:
            return 0
        n = min(self.tick_iters, min(j.req.iters - j.planned for j in jobs))
        b = self._plan(jobs)
        b.step(n, stream=self.stream)
        ev = torch.cuda.Event()
        ev.record(self.stream)
        finishing = []
        for j in jobs:
            j.planned += n
            if j.planned >= j.req.iters:
                finishing.append(j)
        self.inflight.append(Tick(ev, b, jobs, n, finishing))
        self.ticks += 1
        return n

    def _retire(self, t: Tick):
        """Tick t has completed on the GPU: copy the finished jobs' results (on a side stream
        ordered after this tick only), release their memory."""
        t_end = time.perf_counter()
        for j in t.jobs:
            j.done_iters += t.n
        if t.finishing:
            q = {j: t.jobs.index(j) for j in t.finishing}
            with torch.cuda.stream(self.copy_stream):
                self.copy_stream.wait_event(t.event)
                rec = t.batch.records()
                for j in t.finishing:
                    j.last_rd = rec[t.n - 1, q[j]].cpu().numpy()
                    j.final = (j.state.latents.cpu(), j.state.params.cpu())
            for j in t.finishing:
                j.finished = t_end
                if not j.cancelled:
                    self.done[j.req.rid] = j
                self._release(j)
        for j in list(self.active):  # cancelled jobs leave once no queued tick uses them
            if j.cancelled and not any(j in u.jobs for u in self.inflight):
                self._release(j)

    def _retire_ready(self, block: bool = False):
        while self.inflight and (block or self.inflight[0].event.query()):
            t = self.inflight.popleft()
            t.event.synchronize()
            self._retire(t)
            block = False

    def tick(self, now: float) -> int:
        """Synchronous tick: admit what fits, run one tick of all active jobs, retire it.
        Returns the number of iterations run (0 when idle)."""
        self._retire_ready(block=True) if self.inflight else None
        self._admit(now)
        n = self._launch()
        while self.inflight:
            self._retire_ready(block=True)
        return n

    def run(self, requests, t0: float | None = None, max_seconds: float | None = None):
        """Serve (arrival_offset_s, image, lam, seed, iters) requests in real time, with up to
        max_inflight ticks queued on the GPU."""
        t0 = time.perf_counter() if t0 is None else t0
        pending = sorted(requests, key=lambda r: r[0])
        k = 0
        while k < len(pending) or self.queue or self.active or self.inflight:
            now = time.perf_counter()
            while k < len(pending) and t0 + pending[k][0] <= now:
                off, img, lam, seed, iters = pending[k]
                self.submit(img, lam, seed, iters, arrival=t0 + off)
                k += 1
            self._retire_ready()
            self._admit(now)
            if len(self.inflight) < self.max_inflight and self._launch():
                continue
            if self.inflight:
                self._retire_ready(block=True)  # the GPU is busy with everything there is
            elif k < len(pending):
                time.sleep(max(0.0, min(0.005, t0 + pending[k][0] - time.perf_counter())))
            elif self.queue and not self.active:
                continue
            if max_seconds is not None and time.perf_counter() - t0 > max_seconds:
                break
        while self.inflight:
            self._retire_ready(block=True)
        self.batch = None

    def latencies(self):
        return {rid: j.finished - j.req.arrival for rid, j in self.done.items()}


def benchmark(rates=(2.0, 8.0, 32.0), n_requests=64, iters=5000, budget_gb=80.0, tick_iters=50, slots=8,
              seed0=inputs.SEED0):
    out = []
    for rate in rates:
        reqs = []
        for q, (t, (H, W), lam) in enumerate(inputs.serve_requests(rate, n_requests, seed0)):
            img = torch.tensor(inputs.image(H, W, seed=seed0 + 1000 + q, texture_sigma=0.02))
            reqs.append((t, img, lam, seed0 + 7 * q, iters))
        srv = EncodeServer(int(budget_gb * 2 ** 30), tick_iters=tick_iters, slots=slots)
        t0 = time.perf_counter()
        srv.run(reqs, t0=t0)
        wall = time.perf_counter() - t0
        lat = np.array(sorted(srv.latencies().values()))
        pix = sum(r[1].shape[1] * r[1].shape[2] for r in reqs)
        span = max(r[0] for r in reqs) - min(r[0] for r in reqs)
        out.append({
            "rate_offered_per_s": rate, "requests": n_requests, "iters_per_request": iters,
            "offered_requests_per_s": (n_requests - 1) / span if span > 0 else None,
            "offered_mpix_iter_per_s": pix * iters / span / 1e6 if span > 0 else None,
            "served": len(srv.done), "served_requests_per_s": len(srv.done) / wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "min_latency_s": float(lat[0]), "max_latency_s": float(lat[-1]),
            "mpix_iter_per_s": pix * iters / wall / 1e6, "wall_s": wall, "ticks": srv.ticks, "plans": srv.plans,
            "peak_hbm_gb": srv.peak_in_use / 2 ** 30, "budget_gb": budget_gb, "slots": slots,
        })
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", default="2,8,32")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--iters", type=int, default=5000)
    ap.add_argument("--budget-gb", type=float, default=80.0)
    ap.add_argument("--tick-iters", type=int, default=50)
    ap.add_argument("--slots", type=int, default=8, help="jobs running at once at most (0: as many as fit in memory)")
    a = ap.parse_args()
    for line in benchmark(tuple(float(r) for r in a.rates.split(",")), a.requests, a.iters, a.budget_gb, a.tick_iters,
                          a.slots):
        print(json.dumps(line), flush=True)
