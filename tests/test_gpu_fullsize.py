"""Parity at the benchmark's full size and at the extreme shapes the API accepts.

* 512x768 (the timed workload, in the launch configuration the benchmark uses: one encoder
  iteration per call, the workspace entry point): the rate-distortion forward with additive noise
  and the full FP64 gradient of the oracle against the CUDA path (loss, rate and distortion 1e-4
  relative; gradients 1e-3 of each block's largest magnitude), and one encoder iteration against
  the oracle's loss record.
* Rows and columns at the 16384 limit (1 x 16384 and 16384 x 1, where every grid but the finest
  is a single row or column and the replicate clamp acts on every tap of the other axis).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02726_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM = 1e-3
SEED = 77


def _blocks(H, W):
    out, off = [], 0
    for k, (h, w) in enumerate(inputs.grid_shapes(H, W)):
        out.append((f"latents grid {k}", slice(off, off + h * w), True))
        off += h * w
    for name, (po, shape) in inputs.PARAM_OFFSETS.items():
        out.append((name, slice(po, po + int(np.prod(shape))), False))
    return out


def _parity(cc, H, W, img, lat, par, step):
    gi, gl, gp = (torch.tensor(a, device="cuda") for a in (img, lat, par))
    ws = cc.workspace(H, W)
    hp = cc.hparams(lam=LAM, seed=SEED)
    rd = torch.zeros(3, dtype=torch.float64, device="cuda")
    cc.forward(gi, gl, gp, H=H, W=W, hp=hp, step=step, relax=cc.CC_RELAX_NOISE, ws=ws, rd=rd)
    glat, gpar = torch.zeros_like(gl), torch.zeros_like(gp)
    cc.backward(gi, gl, gp, glat, gpar, H=H, W=W, hp=hp, step=step, relax=cc.CC_RELAX_NOISE, ws=ws)
    torch.cuda.synchronize()
    o = oracle.loss_grad(img, lat, par, lam=LAM, mode=oracle.MODE_NOISE, seed=SEED, step=step)
    got = rd.cpu().numpy()
    for k, key in enumerate(("loss", "rate_bits", "mse")):
        assert abs(got[k] - o[key]) <= 1e-4 * abs(o[key]), (key, got[k], o[key])
    gl_, gp_ = glat.double().cpu().numpy(), gpar.double().cpu().numpy()
    for name, sl, is_lat in _blocks(H, W):
        g, ref = (gl_, o["grad_latents"]) if is_lat else (gp_, o["grad_params"])
        scale = np.abs(ref[sl]).max()
        err = np.abs(g[sl] - ref[sl]).max()
        assert err <= 1e-3 * scale + 1e-30, f"{name}: max err {err:.3e}, block max {scale:.3e}"


def test_full_size_forward_and_gradient_match_oracle(cc):
    H, W = 512, 768
    img = inputs.image(H, W, seed=1, texture_sigma=0.02)
    lat, par = inputs.random_state(H, W, seed=2)
    _parity(cc, H, W, img, lat, par, step=3)


def test_full_size_encoder_iteration_matches_oracle(cc):
    """One call of one iteration, as the benchmark times it: the loss record against the oracle's,
    and Adam's first step moving no latent by more than the learning rate (|m / (sqrt(v) + eps)|
    <= 1 at step 1) while moving most of them."""
    H, W = 512, 768
    img = inputs.image(H, W, seed=1, texture_sigma=0.02)
    lat, par = inputs.initial_state(H, W, seed=2)
    gi = torch.tensor(img, device="cuda")
    st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"))
    ws = cc.workspace(H, W)
    rd = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
    cc.encode_step(gi, st, 1, H=H, W=W, hp=cc.hparams(lam=LAM, seed=SEED), ws=ws, rd=rd)
    torch.cuda.synchronize()
    ost = oracle.State(lat, par)
    o = oracle.encode(img, ost, 1, lam=LAM, seed=SEED)
    assert abs(rd[0, 0].item() - o["loss"][0]) <= 1e-4 * abs(o["loss"][0])
    moved = np.abs(st.latents.cpu().numpy().astype(np.float64) - lat.astype(np.float64))
    assert moved.max() <= 1e-2 + 2e-6
    ref_moved = np.abs(ost.latents - lat.astype(np.float64))
    assert abs(np.mean(moved) - np.mean(ref_moved)) <= 1e-3 * np.mean(ref_moved)
    assert int(st.step.item()) == 1


@pytest.mark.parametrize("H,W", [(1, 16384), (16384, 1), (3, 16384)])
def test_extreme_aspect_ratios_match_oracle(cc, H, W):
    img = inputs.image(H, W, seed=H + W)
    lat, par = inputs.random_state(H, W, seed=H * 3 + W)
    _parity(cc, H, W, img, lat, par, step=0)
