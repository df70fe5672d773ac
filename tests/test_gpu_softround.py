"""GPU parity of the paper's training proxy and schedule (Sec. IV-C/D, Eq. 13-14, Table I) against
the FP64 oracle: y~ = s_T(s_T(y) + sigma n) in the main stage with sigma, T linear and the learning
rate cosine over n_main steps; rounding with frozen latents in the hard-round stage.

Tolerances as for the additive proxy: loss, rate and distortion 1e-4 relative, gradients 1e-3 of
each block's largest magnitude, the schedule trajectory 1e-3 relative per iteration.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2605_02726_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM = 1e-2
SEED = 4321
N_MAIN = 40


def _sched(t, n_main=N_MAIN, s0=0.22, s1=0.15, t0=0.35, t1=0.08, lr=1e-2, lr_min=1e-5):
    if t >= n_main:
        return dict(mode=oracle.MODE_HARD, sigma=0.0, temp=1.0, lr=lr_min)
    f = t / n_main
    return dict(mode=oracle.MODE_SOFTROUND, sigma=s0 + (s1 - s0) * f, temp=t0 + (t1 - t0) * f,
                lr=lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * f)))


def _hp(cc):
    return cc.hparams_schedule(lam=LAM, n_main=N_MAIN, seed=SEED)


def _blocks(H, W):
    out, off = [], 0
    for k, (h, w) in enumerate(inputs.grid_shapes(H, W)):
        out.append((f"latents grid {k}", slice(off, off + h * w), True))
        off += h * w
    for name, (po, shape) in inputs.PARAM_OFFSETS.items():
        out.append((name, slice(po, po + int(np.prod(shape))), False))
    return out


@pytest.mark.parametrize("H,W,step", [(64, 64, 0), (37, 53, 17), (64, 64, 39), (40, 24, 40), (33, 65, 55)])
def test_softround_forward_backward_match_oracle(cc, H, W, step):
    img = inputs.image(H, W, seed=H + W)
    lat, par = inputs.random_state(H, W, seed=H * W)
    gi, gl, gp = (torch.tensor(a, device="cuda") for a in (img, lat, par))
    ws = cc.workspace(H, W)
    rd = torch.zeros(3, dtype=torch.float64, device="cuda")
    cc.forward(gi, gl, gp, H=H, W=W, hp=_hp(cc), step=step, relax=cc.CC_RELAX_NOISE, ws=ws, rd=rd)
    glat, gpar = torch.zeros_like(gl), torch.zeros_like(gp)
    cc.backward(gi, gl, gp, glat, gpar, H=H, W=W, hp=_hp(cc), step=step, relax=cc.CC_RELAX_NOISE, ws=ws)
    torch.cuda.synchronize()
    s = _sched(step)
    o = oracle.loss_grad(img, lat, par, lam=LAM, mode=s["mode"], seed=SEED, step=step, sigma=s["sigma"],
                         temp=s["temp"])
    got = rd.cpu().numpy()
    for k, key in enumerate(("loss", "rate_bits", "mse")):
        assert abs(got[k] - o[key]) <= 1e-4 * abs(o[key]), key
    gl_, gp_ = glat.double().cpu().numpy(), gpar.double().cpu().numpy()
    if step >= N_MAIN:
        assert np.all(gl_ == 0.0)  # hard-round stage: no latent gradient
    for name, sl, is_lat in _blocks(H, W):
        g, ref = (gl_, o["grad_latents"]) if is_lat else (gp_, o["grad_params"])
        scale = np.abs(ref[sl]).max()
        assert np.abs(g[sl] - ref[sl]).max() <= 1e-3 * scale + 1e-30, name


def test_schedule_trajectory_and_frozen_latents(cc):
    H = W = 48
    n_main, n_iters = 24, 30
    img = inputs.image(H, W, seed=31)
    lat, par = inputs.initial_state(H, W, seed=32)
    hp = cc.hparams_schedule(lam=LAM, n_main=n_main, seed=SEED)
    st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"))
    gi = torch.tensor(img, device="cuda")
    ws = cc.workspace(H, W)
    rd = torch.zeros(n_iters, 3, dtype=torch.float64, device="cuda")
    cc.encode_step(gi, st, n_main, H=H, W=W, hp=hp, ws=ws, rd=rd[:n_main])
    y_main = st.latents.clone()
    m_main = st.m_lat.clone()
    cc.encode_step(gi, st, n_iters - n_main, H=H, W=W, hp=hp, ws=ws, rd=rd[n_main:])
    torch.cuda.synchronize()
    assert torch.equal(st.latents, y_main) and torch.equal(st.m_lat, m_main)
    ref = oracle.State(lat, par)
    o = oracle.encode_schedule(img, ref, n_iters, lam=LAM, seed=SEED, n_main=n_main)
    got = rd[:, 0].cpu().numpy()
    np.testing.assert_allclose(got, o["loss"], rtol=1e-3)
    assert got[-1] < got[0]


def test_schedule_batch_equals_single(cc):
    sizes = [(40, 56), (24, 24)]
    jobs, singles = [], []
    for q, (H, W) in enumerate(sizes):
        img = torch.tensor(inputs.image(H, W, seed=60 + q), device="cuda")
        lat, par = inputs.initial_state(H, W, seed=70 + q)
        hp = cc.hparams_schedule(lam=LAM, n_main=5, seed=SEED + q)
        jobs.append((img, cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda")), hp))
        singles.append((img, cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda")), hp))
    be = cc.BatchEncoder(jobs, rd_capacity=8)
    be.step(8)
    for img, st, hp in singles:
        H, W = img.shape[1], img.shape[2]
        cc.encode_step(img, st, 8, H=H, W=W, hp=hp, ws=cc.workspace(H, W))
    torch.cuda.synchronize()
    for (_, a, _), (_, b, _) in zip(jobs, singles):
        assert torch.equal(a.latents, b.latents) and torch.equal(a.params, b.params)
    be.close()
