"""A third, test-only formulation of the encoder-step forward in vectorised torch float64.

It is written differently from the oracle on purpose (padding + slicing for the causal context,
a transposed 1-D convolution on a replicate-padded signal for the upsampler, F.conv2d for the
residual convolutions, direct CDF differences for the Laplace mass) so that agreement pins the
oracle's loops, and torch autograd through it pins the oracle's hand-written adjoint.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as F

from paper_2605_02726_gb300 import inputs

CTX = [(0, -1), (-1, 0), (-1, -1), (-1, 1), (0, -2), (-2, 0), (-1, -2), (-1, 2), (-2, -1), (-2, 1),
       (-2, -2), (-2, 2), (0, -3), (-3, 0), (-1, -3), (-1, 3)]
L = 7
P_MIN = 1.0 / 65536.0


def splitmix_noise(seed: int, t: int, n: int) -> np.ndarray:
    """SplitMix64 output function on seed ^ ((t << 32) + i) * gamma, top 24 bits -> [-1/2, 1/2)."""
    M = (1 << 64) - 1
    out = np.empty(n)
    for i in range(n):
        z = (seed ^ ((((t << 32) + i) * 0x9E3779B97F4A7C15) & M)) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        z = z ^ (z >> 31)
        out[i] = (z >> 40) / 16777216.0 - 0.5
    return out


def P(params: torch.Tensor, name: str) -> torch.Tensor:
    o, shape = inputs.PARAM_OFFSETS[name]
    return params[o:o + int(np.prod(shape))].reshape(shape)


def split_grids(lat: torch.Tensor, H: int, W: int, hyper: bool = False):
    out, o = [], 0
    for h, w in inputs.grid_shapes(H, W, hyper=hyper):
        out.append(lat[o:o + h * w].reshape(h, w))
        o += h * w
    return out


def up1d_last(x: torch.Tensor, taps: torch.Tensor, n_out: int) -> torch.Tensor:
    """x2 upsampling along the last axis: transposed conv (stride 2) of the replicate-padded
    signal with h = [a b c d d c b a], output window starting at 7."""
    a, b, c, d = taps[0], taps[1], taps[2], taps[3]
    h = torch.stack([a, b, c, d, d, c, b, a]).reshape(1, 1, 8)
    lead = x.shape[:-1]
    n = x.shape[-1]
    xf = x.reshape(-1, 1, n)
    xp = torch.cat([xf[..., :1], xf[..., :1], xf, xf[..., -1:], xf[..., -1:]], dim=-1)
    y = F.conv_transpose1d(xp, h, stride=2)
    y = y[..., 7:7 + n_out]
    return y.reshape(*lead, n_out)


def upsample2d(x: torch.Tensor, taps: torch.Tensor, th: int, tw: int) -> torch.Tensor:
    r = up1d_last(x, taps, tw)
    return up1d_last(r.transpose(-1, -2), taps, th).transpose(-1, -2)


def laplace_mass(y, mu, b):
    def cdf(z):
        return 0.5 + 0.5 * torch.sign(z) * (1.0 - torch.exp(-torch.abs(z) / b))
    return cdf(y + 0.5 - mu) - cdf(y - 0.5 - mu)


def forward(image: torch.Tensor, yt_flat: torch.Tensor, params: torch.Tensor, lam: float):
    """Returns (loss, rate_bits, mse, mu, logb) from already-relaxed latents yt_flat.  A parameter
    vector of 1451 values carries the hyperlatent IFCE block: the latents then hold three
    hyperlatent grids after the main ones (Sec. III-A3)."""
    _, H, W = image.shape
    hyper = params.shape[0] == inputs.N_PARAMS_H
    grids = split_grids(yt_flat, H, W, hyper)
    shapes = inputs.grid_shapes(H, W, hyper=hyper)
    rate = yt_flat.new_zeros(())
    mus, lbs = [], []
    for k in range(len(shapes)):
        Y = grids[k]
        h, w = shapes[k]
        Yp = F.pad(Y[None, None], (3, 3, 3, 0))[0, 0]
        s = torch.stack([Yp[3 + dy:3 + dy + h, 3 + dx:3 + dx + w] for dy, dx in CTX], dim=-1)
        if k < 3:
            rs = []
            for gj in range(k + 1, L):
                sh = gj - k
                hj, wj = shapes[gj]
                ri = torch.clamp(torch.arange(h) >> sh, max=hj - 1)
                ci = torch.clamp(torch.arange(w) >> sh, max=wj - 1)
                rs.append(grids[gj][ri][:, ci])
            r = torch.stack(rs, dim=-1)
            f = r @ P(params, f"ifce{k}.w").T + P(params, f"ifce{k}.b")
            if hyper:  # the hyperlatent grids (shapes of grids 4, 5, 6) as three more inputs
                hs = []
                for q in range(inputs.N_HYPER_GRIDS):
                    sh = 4 + q - k
                    hj, wj = shapes[L + q]
                    ri = torch.clamp(torch.arange(h) >> sh, max=hj - 1)
                    ci = torch.clamp(torch.arange(w) >> sh, max=wj - 1)
                    hs.append(grids[L + q][ri][:, ci])
                wh = params[inputs.N_PARAMS:].reshape(3, 4, 3)[k]
                f = f + torch.stack(hs, dim=-1) @ wh.T
        else:
            f = s.new_zeros(h, w, 4)
        c = torch.cat([s, f], dim=-1)
        h1 = torch.relu(c @ P(params, "arm.w1").T + P(params, "arm.b1"))
        h2 = torch.relu(h1 @ P(params, "arm.w2").T + P(params, "arm.b2"))
        o = h2 @ P(params, "arm.w3").T + P(params, "arm.b3") + c @ P(params, "arm.ws").T + P(params, "arm.bs")
        mu, logb = o[..., 0], torch.clamp(o[..., 1], -5.0, 5.0)
        p = laplace_mass(Y, mu, torch.exp(logb))
        rate = rate + (-torch.log2(torch.clamp(p, min=P_MIN))).sum()
        mus.append(mu.reshape(-1))
        lbs.append(logb.reshape(-1))
    # upsampling cascade
    S = grids[L - 1][None]
    taps = P(params, "up.taps")
    for m in range(L - 2, -1, -1):
        th, tw = shapes[m]
        S = torch.cat([grids[m][None], upsample2d(S, taps[m], th, tw)], dim=0)
    z = S  # [L, H, W], channel j = grid j
    zz = z.permute(1, 2, 0)
    a = zz @ P(params, "syn.w1").T + P(params, "syn.b1")
    t = (F.gelu(a) @ P(params, "syn.w2").T + P(params, "syn.b2") + zz @ P(params, "syn.ws").T
         + P(params, "syn.bs")).permute(2, 0, 1)

    def res(x, wname, bname):
        xp = F.pad(x[None], (1, 1, 1, 1), mode="replicate")
        return x + F.conv2d(xp, P(params, wname), P(params, bname))[0]

    x1 = res(t, "conv1.w", "conv1.b")
    xh = res(x1, "conv2.w", "conv2.b")
    mse = ((xh - image) ** 2).mean()
    loss = mse + lam * rate / (H * W)
    return loss, rate, mse, torch.cat(mus), torch.cat(lbs), xh


def loss_and_grads(image_np, yt_np, params_np, lam):
    image = torch.tensor(image_np, dtype=torch.float64)
    yt = torch.tensor(yt_np, dtype=torch.float64, requires_grad=True)
    params = torch.tensor(params_np, dtype=torch.float64, requires_grad=True)
    loss, rate, mse, _, _, _ = forward(image, yt, params, lam)
    loss.backward()
    return dict(loss=loss.item(), rate_bits=rate.item(), mse=mse.item(),
                grad_latents=yt.grad.numpy(), grad_params=params.grad.numpy())


def log2e() -> float:
    return 1.0 / math.log(2.0)
