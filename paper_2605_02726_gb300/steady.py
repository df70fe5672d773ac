"""Steady-state encoder iterations for profiling: the 512x768 workload of `bench.py`, its
iterations run back to back in calls of several iterations, with no L2 flush in between (the
state an encode is in between its first and last iteration).  For counter captures such as

  ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --cache-control none ... \\
      python -m paper_2605_02726_gb300.steady

  python -m paper_2605_02726_gb300.steady [--calls 6] [--iters 8] [--H 512] [--W 768]
"""
from __future__ import annotations

import argparse

import torch

from . import inputs
from . import lib as cc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--calls", type=int, default=6)
    ap.add_argument("--iters", type=int, default=8)
    ap.add_argument("--H", type=int, default=512)
    ap.add_argument("--W", type=int, default=768)
    a = ap.parse_args()
    img = torch.tensor(inputs.image(a.H, a.W, seed=inputs.SEED0, texture_sigma=0.02), device="cuda")
    lat, par = inputs.initial_state(a.H, a.W, seed=inputs.SEED0 + 1)
    st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"))
    ws = cc.workspace(a.H, a.W)
    hp = cc.hparams(lam=1e-3, seed=7)
    rd = torch.zeros(a.iters, 3, dtype=torch.float64, device="cuda")
    for _ in range(a.calls):
        cc.encode_step(img, st, a.iters, H=a.H, W=a.W, hp=hp, ws=ws, rd=rd)
    torch.cuda.synchronize()
    print(f"{a.calls} calls of {a.iters} iterations, last loss {rd[-1, 0].item():.6f}")


if __name__ == "__main__":
    main()
