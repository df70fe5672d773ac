"""Hyperlatent grids (Sec. III-A3, Eq. 6) on the CUDA path, against the FP64 oracle.

The architecture flag hyper_grids = 3 adds three grids at 1/16, 1/32, 1/64 of the image, coded by
the ARM and read by the IFCEs of grids 0..2; parity at the stated tolerances (loss, rate,
distortion 1e-4 relative; gradients 1e-3 of each block's largest entry, the hyperlatent grids and
their IFCE weights as blocks of their own; integer decode bit-exact), a batch that mixes jobs with
and without hyperlatents bitwise equal to the single-image path, and the seeded initialisation."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02726_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM, SEED = 1e-2, 77


def _blocks(H, W):
    out, off = [], 0
    for k, (h, w) in enumerate(inputs.grid_shapes(H, W, hyper=True)):
        out.append((f"latents grid {k}", slice(off, off + h * w), True))
        off += h * w
    for name, (po, shape) in inputs.PARAM_OFFSETS.items():
        out.append((name, slice(po, po + int(np.prod(shape))), False))
    out.append(("ifce_h.w", slice(inputs.N_PARAMS, inputs.N_PARAMS_H), False))
    return out


def _parity(cc, H, W, seed, step=2):
    img = inputs.image(H, W, seed=seed)
    lat, par = inputs.random_state(H, W, seed=seed + 1, hyper=True)
    assert par.shape[0] == inputs.N_PARAMS_H and lat.shape[0] == inputs.latent_count(H, W, True)
    gi, gl, gp = (torch.tensor(a, device="cuda") for a in (img, lat, par))
    ws = cc.workspace(H, W, hyper=True)
    hp = cc.hparams(lam=LAM, seed=SEED)
    rd = torch.zeros(3, dtype=torch.float64, device="cuda")
    cc.forward(gi, gl, gp, H=H, W=W, hp=hp, step=step, relax=cc.CC_RELAX_NOISE, ws=ws, rd=rd)
    glat, gpar = torch.zeros_like(gl), torch.zeros_like(gp)
    cc.backward(gi, gl, gp, glat, gpar, H=H, W=W, hp=hp, step=step, relax=cc.CC_RELAX_NOISE, ws=ws)
    torch.cuda.synchronize()
    o = oracle.loss_grad(img, lat, par, lam=LAM, mode=oracle.MODE_NOISE, seed=SEED, step=step)
    # The rate's gradient is discontinuous where a latent's mass P crosses the 2^-16 floor; a state
    # with a latent within FP32 reach of it has no gradient parity to check there.
    f = oracle.forward(img, lat, par, lam=LAM, mode=oracle.MODE_NOISE, seed=SEED, step=step, per_latent=True)
    yt = lat.astype(np.float64) + oracle.noise(SEED, step, lat.shape[0])
    b = np.exp(f["logb"])

    def cdf(z):
        return 0.5 + 0.5 * np.sign(z) * (1.0 - np.exp(-np.abs(z) / b))

    mass = cdf(yt + 0.5 - f["mu"]) - cdf(yt - 0.5 - f["mu"])
    assert np.abs(mass / 2.0 ** -16 - 1.0).min() > 1e-4, "a latent sits on the 2^-16 floor: pick another seed"
    got = rd.cpu().numpy()
    for k, key in enumerate(("loss", "rate_bits", "mse")):
        assert abs(got[k] - o[key]) <= 1e-4 * abs(o[key]), (key, got[k], o[key])
    gl_, gp_ = glat.double().cpu().numpy(), gpar.double().cpu().numpy()
    for name, sl, is_lat in _blocks(H, W):
        g, ref = (gl_, o["grad_latents"]) if is_lat else (gp_, o["grad_params"])
        scale = np.abs(ref[sl]).max()
        err = np.abs(g[sl] - ref[sl]).max()
        assert err <= 1e-3 * scale + 1e-30, f"{name}: max err {err:.3e}, block max {scale:.3e}"


@pytest.mark.parametrize("H,W,seed", [(64, 64, 192), (37, 53, 143), (130, 67, 264), (16, 16, 48), (512, 768, 2049)])
def test_hyper_forward_and_gradient_match_oracle(cc, H, W, seed):
    _parity(cc, H, W, seed=seed)


@pytest.mark.parametrize("H,W", [(64, 64), (45, 77), (512, 768)])
def test_hyper_decode_bit_exact(cc, H, W):
    q = inputs.quantized_latents(H, W, seed=H + 3 * W, hyper=True)
    _, par = inputs.random_state(H, W, seed=H * W + 1, hyper=True)
    ws = cc.workspace(H, W, hyper=True)
    N = q.shape[0]
    gq, gp = torch.tensor(q, device="cuda"), torch.tensor(par, device="cuda")
    prob, mu, lb = (torch.zeros(N, dtype=torch.int32, device="cuda") for _ in range(3))
    img = torch.zeros(3, H, W, device="cuda")
    cc.decode_image(gq, gp, H=H, W=W, ws=ws, image_out=img, prob=prob, mu_q=mu, logb_q=lb)
    torch.cuda.synchronize()
    o = oracle.decode_probs(H, W, q, par)
    np.testing.assert_array_equal(mu.cpu().numpy(), o["mu_q"])
    np.testing.assert_array_equal(lb.cpu().numpy(), o["logb_q"])
    np.testing.assert_array_equal(prob.cpu().numpy().view(np.uint32), o["prob_q16"])
    np.testing.assert_allclose(img.cpu().numpy(), oracle.decode_image(H, W, q, par), rtol=0, atol=1e-4)


def test_hyper_encode_iterations_and_mixed_batch(cc):
    """Three iterations with hyperlatents: the loss record against the oracle's encode; a batch of
    a job with and a job without hyperlatents, each bitwise the single-image path."""
    H, W = 48, 64
    img = inputs.image(H, W, seed=5)
    lat, par = inputs.initial_state(H, W, seed=6, hyper=True)
    gi = torch.tensor(img, device="cuda")
    st = cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda"))
    rd = torch.zeros(3, 3, dtype=torch.float64, device="cuda")
    hp = cc.hparams(lam=LAM, seed=SEED)
    cc.encode_step(gi, st, 3, H=H, W=W, hp=hp, ws=cc.workspace(H, W, hyper=True), rd=rd)
    torch.cuda.synchronize()
    ost = oracle.State(lat, par)
    o = oracle.encode(img, ost, 3, lam=LAM, seed=SEED)
    np.testing.assert_allclose(rd[:, 0].cpu().numpy(), o["loss"], rtol=1e-4)

    lat2, par2 = inputs.initial_state(40, 24, seed=8)
    img2 = torch.tensor(inputs.image(40, 24, seed=9), device="cuda")
    jobs = [(gi, cc.EncoderState(torch.tensor(lat, device="cuda"), torch.tensor(par, device="cuda")), hp),
            (img2, cc.EncoderState(torch.tensor(lat2, device="cuda"), torch.tensor(par2, device="cuda")), hp)]
    singles = []
    for im, s0, h in jobs:
        s = s0.clone()
        Hh, Ww = im.shape[1], im.shape[2]
        cc.encode_step(im, s, 2, H=Hh, W=Ww, hp=h, ws=cc.workspace(Hh, Ww, hyper=s.params.numel() == cc.N_PARAMS_H))
        singles.append(s)
    be = cc.BatchEncoder(jobs, rd_capacity=2)
    be.step(2)
    torch.cuda.synchronize()
    for (_, s, _), r in zip(jobs, singles):
        assert torch.equal(s.latents, r.latents) and torch.equal(s.params, r.params)
    be.close()


def test_hyper_init_state(cc):
    """The seeded device initialisation covers the hyperlatents (0.01 times the normal at step
    -1, like every latent) and the hyperlatent IFCE weights (2u / sqrt(fan_in), the fan-in of an
    IFCE counting its three hyperlatent inputs)."""
    H, W, seed = 40, 56, 3
    st = cc.EncoderState.init(H, W, seed, hyper=True)
    torch.cuda.synchronize()
    n = inputs.latent_count(H, W, True)
    assert st.latents.numel() == n and st.params.numel() == inputs.N_PARAMS_H
    np.testing.assert_allclose(st.latents.cpu().numpy().astype(np.float64), 0.01 * oracle.gauss(seed, -1, n),
                               rtol=1e-5, atol=5e-6)
    u = oracle.noise(seed, -2, inputs.N_PARAMS_H).astype(np.float32)
    p = st.params.cpu().numpy()
    for k, (name, nin) in enumerate((("ifce0.w", 6), ("ifce1.w", 5), ("ifce2.w", 4))):
        o, shape = inputs.PARAM_OFFSETS[name]
        fan = np.sqrt(np.float32(nin + 3))
        np.testing.assert_allclose(p[o:o + 4 * nin], 2 * u[o:o + 4 * nin] / fan, rtol=1e-6)
        oh = inputs.N_PARAMS + 12 * k
        np.testing.assert_allclose(p[oh:oh + 12], 2 * u[oh:oh + 12] / fan, rtol=1e-6)
