"""Pins of the oracle's hyperlatent grids (Sec. III-A3, Eq. 6) against facts outside it: the
independent float64 torch composition (forward) and its autograd (adjoint), central differences,
and what the paper states about hyperlatents -- they are entropy coded by the same ARM, read only
by the IFCEs, and never reach the synthesis."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02726_gb300 import inputs
from tests import torch_ref

SHAPES = [(16, 16), (24, 40), (37, 21)]


def _state(H, W, seed):
    img = inputs.image(H, W, seed=seed).astype(np.float64)
    lat, par = inputs.random_state(H, W, seed=seed + 1, hyper=True)
    return img, lat.astype(np.float64), par.astype(np.float64)


def test_hyper_geometry():
    H, W = 37, 21
    shapes = oracle.grid_shapes(H, W, hyper=True)
    assert shapes == inputs.grid_shapes(H, W, hyper=True)
    assert shapes[7:] == shapes[4:7]  # b = 4: 1/16, 1/32, 1/64
    assert oracle.latent_count(H, W, True) == oracle.latent_count(H, W) + sum(h * w for h, w in shapes[4:7])


@pytest.mark.parametrize("H,W", SHAPES)
def test_hyper_forward_matches_torch_composition(H, W):
    img, yt, par = _state(H, W, 30 + H)
    o = oracle.forward(img, yt, par, lam=1e-2, mode=oracle.MODE_IDENTITY, per_latent=True)
    loss, rate, mse, mu, logb, xh = torch_ref.forward(torch.tensor(img), torch.tensor(yt), torch.tensor(par), 1e-2)
    assert abs(o["loss"] - loss.item()) <= 1e-12 * abs(loss.item())
    assert abs(o["rate_bits"] - rate.item()) <= 1e-11 * abs(rate.item())
    np.testing.assert_allclose(o["mu"], mu.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(o["logb"], logb.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(o["xhat"], xh.numpy(), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("H,W", SHAPES)
def test_hyper_adjoint_matches_torch_autograd(H, W):
    img, yt, par = _state(H, W, 40 + W)
    o = oracle.loss_grad(img, yt, par, lam=3e-2, mode=oracle.MODE_IDENTITY)
    r = torch_ref.loss_and_grads(img, yt, par, 3e-2)
    assert abs(o["loss"] - r["loss"]) <= 1e-12 * abs(r["loss"])
    for key in ("grad_latents", "grad_params"):
        a, b = o[key], r[key]
        assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max(), key
    n_main = oracle.latent_count(H, W)
    assert np.abs(o["grad_latents"][n_main:]).max() > 0  # the hyperlatents are trained
    assert np.abs(o["grad_params"][inputs.N_PARAMS:]).max() > 0


def test_hyperlatents_reach_the_rate_but_never_the_reconstruction():
    H, W = 24, 40
    img, yt, par = _state(H, W, 5)
    base = oracle.forward(img, yt, par, lam=1e-2, mode=oracle.MODE_IDENTITY, per_latent=True)
    n_main = oracle.latent_count(H, W)
    for i in (n_main, n_main + 3, yt.shape[0] - 1):
        y2 = yt.copy()
        y2[i] += 1.7
        o = oracle.forward(img, y2, par, lam=1e-2, mode=oracle.MODE_IDENTITY, per_latent=True)
        np.testing.assert_array_equal(o["xhat"], base["xhat"])
        assert o["mse"] == base["mse"]
        assert o["rate_bits"] != base["rate_bits"]
        # the main grids that read it through their IFCE see it; grids 3..6 never do
        offs = np.cumsum([0] + [h * w for h, w in oracle.grid_shapes(H, W)])
        np.testing.assert_array_equal(o["mu"][offs[3]:n_main], base["mu"][offs[3]:n_main])
        assert np.any(o["mu"][:offs[3]] != base["mu"][:offs[3]])


def test_zero_hyper_weights_leave_the_main_entropy_model_unchanged():
    """With the hyperlatent IFCE block at zero, every main latent's (mu, log b) is the model's
    without hyperlatents, and the rate grows by the bits of the hyperlatents, which the ARM codes
    from their spatial context alone."""
    H, W = 24, 40
    img, yt, par = _state(H, W, 9)
    par[inputs.N_PARAMS:] = 0.0
    n_main = oracle.latent_count(H, W)
    h = oracle.forward(img, yt, par, lam=1e-2, mode=oracle.MODE_IDENTITY, per_latent=True)
    p = oracle.forward(img, yt[:n_main], par[:inputs.N_PARAMS], lam=1e-2, mode=oracle.MODE_IDENTITY,
                       per_latent=True)
    np.testing.assert_array_equal(h["mu"][:n_main], p["mu"])
    np.testing.assert_array_equal(h["logb"][:n_main], p["logb"])
    assert h["mse"] == p["mse"]
    assert abs(h["rate_bits"] - p["rate_bits"] - h["bits"][n_main:].sum()) <= 1e-10 * h["rate_bits"]


def test_hyper_gradient_matches_central_differences():
    H, W = 40, 48  # 14 hyperlatents
    img, yt, par = _state(H, W, 61)
    lam = 2e-2
    g = oracle.loss_grad(img, yt, par, lam=lam, mode=oracle.MODE_IDENTITY)
    n_main = oracle.latent_count(H, W)

    def f(y, p):
        return oracle.forward(img, y, p, lam=lam, mode=oracle.MODE_IDENTITY)["loss"]

    coords = [("lat", i) for i in range(n_main, yt.shape[0])]
    coords += [("par", i) for i in range(inputs.N_PARAMS, par.shape[0])]
    checked = 0
    for kind, i in coords:
        def fd(hh):
            y2, p2 = yt.copy(), par.copy()
            arr = y2 if kind == "lat" else p2
            arr[i] += hh
            fp = f(y2, p2)
            arr[i] -= 2 * hh
            return (fp - f(y2, p2)) / (2 * hh)

        d1, d2 = fd(1e-4), fd(5e-5)
        an = (g["grad_latents"] if kind == "lat" else g["grad_params"])[i]
        scale = max(abs(an), 1e-7)
        if abs(d1 - d2) > 1e-6 * scale:  # a kink inside the step
            continue
        checked += 1
        assert abs(d1 - an) <= 1e-5 * scale + 1e-11, (kind, i, d1, an)
    # a hyperlatent feeds every IFCE position under it, so a ReLU kink inside the step is common
    assert checked >= 25


def test_hyper_decode_probabilities_within_their_bounds():
    """The integer decoder with hyperlatents: P_q16 within 8 of 65536 times the Laplace mass of its
    own integer parameters, and the integer ARM within its floor bound of the FP64 ARM on
    2^-8-grid weights (the pins of the decoder without hyperlatents, with the extra inputs)."""
    H, W = 24, 40
    q = inputs.quantized_latents(H, W, seed=43, hyper=True)
    _, par = inputs.random_state(H, W, seed=44, hyper=True)
    d = oracle.decode_probs(H, W, q, par)
    mu = d["mu_q"].astype(np.float64) / 256.0
    b = np.exp(d["logb_q"].astype(np.float64) / 256.0)

    def cdf(z):
        return 0.5 + 0.5 * np.sign(z) * (1.0 - np.exp(-np.abs(z) / b))

    mass = cdf(q + 0.5 - mu) - cdf(q - 0.5 - mu)
    assert np.abs(d["prob_q16"].astype(np.float64) - 65536.0 * mass).max() <= 8.0
    pq = np.rint(par.astype(np.float64) * 256.0) / 256.0
    fl = oracle.forward(np.zeros((3, H, W)), q.astype(np.float64), pq, lam=0.0, mode=oracle.MODE_IDENTITY,
                        per_latent=True)
    W2 = torch_ref.P(torch.tensor(pq), "arm.w2").numpy()
    W3 = torch_ref.P(torch.tensor(pq), "arm.w3").numpy()
    u = 2.0 ** -8
    e_out = u + np.abs(W3) @ (u + np.abs(W2) @ np.full(16, u))
    assert np.abs(d["mu_q"] / 256.0 - fl["mu"]).max() <= e_out[0] + 1e-12
    assert np.abs(d["logb_q"] / 256.0 - fl["logb"]).max() <= e_out[1] + 1e-12
