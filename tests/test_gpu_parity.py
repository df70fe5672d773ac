"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (the stated contract): loss, rate and distortion 1e-4 relative; gradients 1e-3
relative to the largest magnitude of their block (latents per grid, parameters per block);
quantised latents and integer decode probabilities bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02726_gb300 import inputs

pytestmark = pytest.mark.gpu

LAM = 1e-2
SEED = 1234


def _setup(H, W, seed, random=True):
    img = inputs.image(H, W, seed=seed)
    lat, par = (inputs.random_state if random else inputs.initial_state)(H, W, seed=seed + 1)
    return img, lat, par


def _cuda(*arrs):
    return [torch.tensor(a, device="cuda").contiguous() for a in arrs]


def _gpu_forward(cc, img, lat, par, H, W, step, relax, store=False, lam=LAM):
    ws = cc.workspace(H, W, store_activations=store)
    gi, gl, gp = _cuda(img, lat, par)
    rd = torch.zeros(3, dtype=torch.float64, device="cuda")
    xh = torch.zeros(3, H, W, device="cuda")
    cc.forward(gi, gl, gp, H=H, W=W, hp=cc.hparams(lam=lam, seed=SEED), step=step, relax=relax, ws=ws,
               store=store, rd=rd, xhat=xh)
    torch.cuda.synchronize()
    return rd.cpu().numpy(), xh.cpu().numpy(), (ws, gi, gl, gp)


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-30)


SHAPES = [(64, 64), (37, 53), (8, 8), (1, 1), (3, 5), (130, 67)]


@pytest.mark.parametrize("H,W", SHAPES)
@pytest.mark.parametrize("relax", [0, 1])
def test_forward_matches_oracle(cc, H, W, relax):
    img, lat, par = _setup(H, W, 10 + H + W)
    rd, xh, _ = _gpu_forward(cc, img, lat, par, H, W, step=5, relax=relax)
    o = oracle.forward(img, lat, par, lam=LAM, mode=relax, seed=SEED, step=5, per_latent=True)
    assert _rel(rd[0], o["loss"]) < 1e-4
    assert _rel(rd[1], o["rate_bits"]) < 1e-4
    assert _rel(rd[2], o["mse"]) < 1e-4
    np.testing.assert_allclose(xh, o["xhat"], rtol=0, atol=2e-4 * max(1.0, np.abs(o["xhat"]).max()))


def _block_check(name, g, ref, tol=1e-3):
    scale = np.abs(ref).max()
    if scale == 0:
        assert np.abs(g).max() == 0, name
        return
    err = np.abs(g - ref).max() / scale
    assert err < tol, f"{name}: max err {err:.2e} relative to block max {scale:.3e}"


def _compare_grads(H, W, gl, gp, o):
    shapes = inputs.grid_shapes(H, W)
    off = 0
    for k, (h, w) in enumerate(shapes):
        _block_check(f"latents grid {k}", gl[off:off + h * w], o["grad_latents"][off:off + h * w])
        off += h * w
    for name, (po, shape) in inputs.PARAM_OFFSETS.items():
        n = int(np.prod(shape))
        _block_check(name, gp[po:po + n], o["grad_params"][po:po + n])


@pytest.mark.parametrize("H,W", [(64, 64), (37, 53), (8, 8), (3, 5), (130, 67)])
@pytest.mark.parametrize("use_stored", [False, True])
def test_backward_matches_oracle(cc, H, W, use_stored):
    img, lat, par = _setup(H, W, 20 + H * W)
    step = 2
    _, _, (ws, gi, glat, gpar) = _gpu_forward(cc, img, lat, par, H, W, step=step, relax=0, store=use_stored)
    gl = torch.zeros_like(glat)
    gp = torch.zeros_like(gpar)
    cc.backward(gi, glat, gpar, gl, gp, H=H, W=W, hp=cc.hparams(lam=LAM, seed=SEED), step=step, relax=0,
                ws=ws, use_stored=use_stored)
    torch.cuda.synchronize()
    o = oracle.loss_grad(img, lat, par, lam=LAM, mode=0, seed=SEED, step=step)
    _compare_grads(H, W, gl.cpu().numpy(), gp.cpu().numpy(), o)


def test_backward_hard_mode_zero_latent_gradient(cc):
    H, W = 32, 48
    img, lat, par = _setup(H, W, 3)
    _, _, (ws, gi, glat, gpar) = _gpu_forward(cc, img, lat, par, H, W, step=0, relax=1)
    gl = torch.ones_like(glat)
    gp = torch.zeros_like(gpar)
    cc.backward(gi, glat, gpar, gl, gp, H=H, W=W, hp=cc.hparams(lam=LAM, seed=SEED), step=0, relax=1, ws=ws)
    torch.cuda.synchronize()
    assert not torch.any(gl)
    o = oracle.loss_grad(img, lat, par, lam=LAM, mode=1)
    for name, (po, shape) in inputs.PARAM_OFFSETS.items():
        n = int(np.prod(shape))
        _block_check(name, gp.cpu().numpy()[po:po + n], o["grad_params"][po:po + n])


def test_encode_step_is_backward_plus_adam(cc):
    """One fused iteration equals coolchic_backward followed by Adam (FP64 on the host)."""
    H, W = 48, 40
    img, lat, par = _setup(H, W, 7)
    hp = cc.hparams(lam=LAM, seed=SEED)
    gi, gl0, gp0 = _cuda(img, lat, par)
    ws = cc.workspace(H, W)
    st = cc.EncoderState(gl0, gp0, step=4)
    rd = torch.zeros(1, 3, dtype=torch.float64, device="cuda")
    cc.encode_step(gi, st, 1, H=H, W=W, hp=hp, ws=ws, rd=rd)
    gl = torch.zeros_like(gl0)
    gp = torch.zeros_like(gp0)
    cc.backward(gi, gl0, gp0, gl, gp, H=H, W=W, hp=hp, step=4, relax=0, ws=ws)
    torch.cuda.synchronize()
    assert int(st.step.item()) == 5
    fr, _, _ = _gpu_forward(cc, img, lat, par, H, W, step=4, relax=0)
    assert _rel(rd[0, 0].item(), fr[0]) < 1e-6
    for p0, g, p1 in ((lat, gl, st.latents), (par, gp, st.params)):
        g = g.double().cpu().numpy()
        m = 0.1 * g
        v = 0.001 * g * g
        t = 5
        ref = p0.astype(np.float64) - 1e-2 * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
        np.testing.assert_allclose(p1.cpu().numpy(), ref, rtol=0, atol=2e-6 + 1e-6 * np.abs(ref).max())


def test_encode_trajectory_config0(cc):
    """64x64, initial state, lambda 1e-3, lr 1e-2, 100 iterations: loss curve vs the FP64 oracle
    (a trajectory check: FP32 and FP64 iterates may drift apart legitimately)."""
    H = W = 64
    img = inputs.image(H, W, seed=inputs.SEED0)
    lat, par = inputs.initial_state(H, W, seed=inputs.SEED0 + 1)
    n = 100
    hp = cc.hparams(lam=1e-3, seed=SEED)
    gi, gl, gp = _cuda(img, lat, par)
    st = cc.EncoderState(gl, gp)
    ws = cc.workspace(H, W)
    rd = torch.zeros(n, 3, dtype=torch.float64, device="cuda")
    cc.encode_step(gi, st, n, H=H, W=W, hp=hp, ws=ws, rd=rd)
    torch.cuda.synchronize()
    ost = oracle.State(lat, par)
    o = oracle.encode(img, ost, n, lam=1e-3, seed=SEED)
    g = rd.cpu().numpy()
    rel = np.abs(g[:, 0] - o["loss"]) / np.abs(o["loss"])
    assert rel.max() < 1e-3, rel.max()
    assert g[-1, 0] < 0.5 * g[0, 0]  # it trains


def test_rate_distortion_hard_matches_oracle(cc):
    H, W = 96, 72
    img, lat, par = _setup(H, W, 99)
    gi, gl, gp = _cuda(img, lat, par)
    ws = cc.workspace(H, W)
    r = cc.rate_distortion(gi, gl, gp, H=H, W=W, hp=cc.hparams(lam=LAM), relax=1, ws=ws)
    o = oracle.forward(img, lat, par, lam=LAM, mode=oracle.MODE_HARD)
    assert _rel(r["loss"], o["loss"]) < 1e-4 and _rel(r["rate_bits"], o["rate_bits"]) < 1e-4


@pytest.mark.parametrize("H,W", [(64, 64), (45, 77), (1, 1), (16, 5), (512, 768)])
def test_decode_bit_exact(cc, H, W):
    q = inputs.quantized_latents(H, W, seed=H + 3 * W)
    _, par = inputs.random_state(H, W, seed=H * W + 1)
    ws = cc.workspace(H, W)
    gq = torch.tensor(q, device="cuda")
    gp = torch.tensor(par, device="cuda")
    N = q.shape[0]
    prob = torch.zeros(N, dtype=torch.int32, device="cuda")
    mu = torch.zeros(N, dtype=torch.int32, device="cuda")
    lb = torch.zeros(N, dtype=torch.int32, device="cuda")
    img = torch.zeros(3, H, W, device="cuda")
    cc.decode_image(gq, gp, H=H, W=W, ws=ws, image_out=img, prob=prob, mu_q=mu, logb_q=lb)
    torch.cuda.synchronize()
    o = oracle.decode_probs(H, W, q, par)
    np.testing.assert_array_equal(mu.cpu().numpy(), o["mu_q"])
    np.testing.assert_array_equal(lb.cpu().numpy(), o["logb_q"])
    np.testing.assert_array_equal(prob.cpu().numpy().view(np.uint32), o["prob_q16"])
    ref = oracle.decode_image(H, W, q, par)
    np.testing.assert_allclose(img.cpu().numpy(), ref, rtol=0, atol=1e-4)


def test_hard_quantisation_bit_exact(cc):
    """The relaxed latents under CC_RELAX_HARD are rint(y) of the FP32 values, ties to even."""
    H, W = 40, 40
    img, lat, par = _setup(H, W, 5)
    lat[:6] = [0.5, 1.5, 2.5, -0.5, -1.5, 3.4999998]
    _, _, (ws, gi, gl, gp) = _gpu_forward(cc, img, lat, par, H, W, step=0, relax=1)
    N = lat.shape[0]
    yt = ws[:N * 4].view(torch.float32)  # first workspace buffer holds y~
    np.testing.assert_array_equal(yt.cpu().numpy(), np.rint(lat.astype(np.float64)).astype(np.float32))


def test_repeat_runs_bitwise_identical(cc):
    H, W = 70, 90
    img, lat, par = _setup(H, W, 11)
    outs = []
    for _ in range(2):
        gi, gl0, gp0 = _cuda(img, lat, par)
        st = cc.EncoderState(gl0, gp0)
        ws = cc.workspace(H, W)
        cc.encode_step(gi, st, 3, H=H, W=W, hp=cc.hparams(lam=LAM, seed=SEED), ws=ws)
        torch.cuda.synchronize()
        outs.append((st.latents.cpu().numpy(), st.params.cpu().numpy()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
