"""Multi-stage encoding (Sec. IV-D, Table I): warm-up candidates in one batch, ranked by their
rate-distortion cost with rounded latents; main stage on the soft-round schedule; hard-round stage.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02726_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM = 1e-2


def test_warmup_keeps_the_best_candidates(cc):
    from paper_2605_02726_gb300 import encoder
    H, W = 40, 56
    img = torch.tensor(inputs.image(H, W, seed=81), device="cuda")
    rounds = ((3, 12), (2, 12))
    best, rankings = encoder.warmup(img, LAM, rounds=rounds, seed=5)
    # the same candidates trained alone: identical states (a job's bits do not depend on the batch)
    alone = {}
    for c in range(3):
        lat, par = inputs.initial_state(H, W, seed=5 + c)
        st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"), soap=True)
        hp = cc.hparams_schedule(lam=LAM, n_main=1 << 40, lr=1e-2, lr_min=1e-2, sigma0=0.22, sigma1=0.22,
                                 temp0=0.35, temp1=0.35, seed=5 + 1000 + c, soap=True)
        cc.encode_step(img, st, 12, H=H, W=W, hp=hp, ws=cc.workspace(H, W))
        alone[c] = (st, hp)
    first = sorted(range(3), key=lambda c: (encoder.rd_hard(img, alone[c][0], LAM)[0], c))
    assert [c for c, _ in rankings[0]] == first
    # the ranking's costs are the FP64 oracle's rate-distortion cost with rounded latents (Eq. 10 at
    # Eq. 12's quantised latents) of each candidate's trained state
    img_np = img.cpu().numpy()
    for c, loss in rankings[0]:
        st = alone[c][0]
        o = oracle.forward(img_np, st.latents.cpu().numpy(), st.params.cpu().numpy(), lam=LAM,
                           mode=oracle.MODE_HARD)
        assert abs(loss - o["loss"]) <= 1e-4 * abs(o["loss"]), (c, loss, o["loss"])
    for c in first[:2]:
        st, hp = alone[c]
        cc.encode_step(img, st, 12, H=H, W=W, hp=hp, ws=cc.workspace(H, W))
    second = sorted(first[:2], key=lambda c: (encoder.rd_hard(img, alone[c][0], LAM)[0], c))
    assert [c for c, _ in rankings[1]] == second
    winner = alone[second[0]][0]
    torch.cuda.synchronize()
    assert torch.equal(best.latents, winner.latents) and torch.equal(best.params, winner.params)
    losses = [l for _, l in rankings[1]]
    assert losses == sorted(losses)


def test_three_stage_encode(cc):
    from paper_2605_02726_gb300 import encoder
    H, W = 48, 64
    img = torch.tensor(inputs.image(H, W, seed=91), device="cuda")
    out = encoder.encode(img, LAM, n_main=30, n_hard=6, rounds=((2, 8), (1, 8)), seed=3, chunk=7)
    rec = out["records"]
    assert rec.shape == (36, 3) and np.all(np.isfinite(rec))
    assert rec[29, 0] < rec[0, 0]                       # the main stage lowers the training loss
    loss, rate, mse = out["rd_hard"]
    assert np.isfinite(loss) and loss > 0 and rate > 0 and mse > 0
    assert abs(loss - (mse + LAM * rate / (H * W))) < 1e-9 * loss
    assert int(out["state"].step.item()) == 36
