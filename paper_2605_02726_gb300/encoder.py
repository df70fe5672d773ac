"""Multi-stage encoding of one image (Sec. IV-D, Table I) on the library's encoder steps.

  1. Warm-up: random initialisations compete; each round trains the surviving candidates for a
     few hundred iterations in one batched launch set (one CUDA launch per kernel for all of
     them), ranks them by their rate-distortion cost with rounded latents (Eq. 10 at Eq. 12's
     quantised latents) and keeps the best (Table I: 5 candidates, then 2, 400 iterations each).
     Candidates train with the soft-round proxy held at the main stage's initial sigma, T and
     learning rate.
  2. Main stage: the selected candidate, with a fresh optimizer state, follows the soft-round
     schedule (sigma and T linear, learning rate cosine) for n_main iterations.
  3. Hard-round stage: n_hard iterations with rounded latents, the latents frozen and the
     parameters at the final learning rate.

The network parameters follow SOAP and the latents Adam (Sec. IV-B) unless soap=False.

`encode(image, lam, ...)` returns the final state, the per-iteration training records of stages 2
and 3, the warm-up ranking and the final rate-distortion cost with rounded latents.
"""
from __future__ import annotations

import numpy as np
import torch

from . import inputs
from . import lib as cc


def _fresh(st: cc.EncoderState) -> cc.EncoderState:
    """Same latents and parameters, zero optimizer moments, step 0."""
    return cc.EncoderState(st.latents.clone(), st.params.clone(), step=0, soap=st.soap is not None)


def rd_hard(image: torch.Tensor, st: cc.EncoderState, lam: float, ws=None):
    """(loss, rate_bits, mse) with rounded latents."""
    H, W = int(image.shape[1]), int(image.shape[2])
    ws = cc.workspace(H, W, device=image.device) if ws is None else ws
    r = cc.rate_distortion(image, st.latents, st.params, H=H, W=W, hp=cc.hparams(lam=lam), relax=cc.CC_RELAX_HARD,
                           ws=ws)
    return r["loss"], r["rate_bits"], r["mse"]


def warmup(image: torch.Tensor, lam: float, *, rounds=((5, 400), (2, 400)), seed: int = 0, lr: float = 1e-2,
           sigma: float = 0.22, temp: float = 0.35, soap: bool = True):
    """Runs the warm-up rounds; returns (best state, per-round rankings [(candidate id, loss)]).

    rounds: (number of candidates entering the round, iterations).  Candidate c starts from
    inputs.initial_state(H, W, seed + c)."""
    H, W = int(image.shape[1]), int(image.shape[2])
    dev = image.device
    n0 = rounds[0][0]
    cands = []
    for c in range(n0):
        lat, par = inputs.initial_state(H, W, seed=seed + c)
        cands.append((c, cc.EncoderState(torch.tensor(lat, device=dev), torch.tensor(par, device=dev), soap=soap)))
    # the main stage's initial proxy, held constant: sigma0 = sigma1, T0 = T1, lr = lr_min
    hp_of = lambda c: cc.hparams_schedule(lam=lam, n_main=1 << 40, lr=lr, lr_min=lr, sigma0=sigma, sigma1=sigma,
                                          temp0=temp, temp1=temp, seed=seed + 1000 + c, soap=soap)
    ws = [cc.workspace(H, W, device=dev) for _ in range(n0)]
    rankings = []
    for n_in, iters in rounds:
        cands = cands[:n_in]
        be = cc.BatchEncoder([(image, st, hp_of(c)) for c, st in cands], rd_capacity=0, workspaces=ws[:len(cands)])
        be.step(iters)
        be.close()
        scored = sorted(((rd_hard(image, st, lam, ws[0])[0], c, st) for c, st in cands), key=lambda x: (x[0], x[1]))
        rankings.append([(c, loss) for loss, c, _ in scored])
        cands = [(c, st) for _, c, st in scored]
    return cands[0][1], rankings


def encode(image: torch.Tensor, lam: float, *, n_main: int, n_hard: int, rounds=((5, 400), (2, 400)),
           seed: int = 0, lr: float = 1e-2, lr_min: float = 1e-5, sigma=(0.22, 0.15), temp=(0.35, 0.08),
           chunk: int = 1000, soap: bool = True):
    """The three stages; returns dict(state, records [n_main + n_hard, 3], warmup, rd_hard)."""
    H, W = int(image.shape[1]), int(image.shape[2])
    dev = image.device
    if rounds:
        best, ranking = warmup(image, lam, rounds=rounds, seed=seed, lr=lr, sigma=sigma[0], temp=temp[0], soap=soap)
        st = _fresh(best)
    else:
        lat, par = inputs.initial_state(H, W, seed=seed)
        st = cc.EncoderState(torch.tensor(lat, device=dev), torch.tensor(par, device=dev), soap=soap)
        ranking = []
    hp = cc.hparams_schedule(lam=lam, n_main=n_main, lr=lr, lr_min=lr_min, sigma0=sigma[0], sigma1=sigma[1],
                             temp0=temp[0], temp1=temp[1], seed=seed, soap=soap)
    ws = cc.workspace(H, W, device=dev)
    total = n_main + n_hard
    rec = torch.zeros(max(total, 1), 3, dtype=torch.float64, device=dev)
    done = 0
    while done < total:
        n = min(chunk, total - done)
        cc.encode_step(image, st, n, H=H, W=W, hp=hp, ws=ws, rd=rec[done:done + n])
        done += n
    torch.cuda.synchronize(dev)
    return dict(state=st, records=rec[:total].cpu().numpy(), warmup=ranking, rd_hard=rd_hard(image, st, lam, ws))
