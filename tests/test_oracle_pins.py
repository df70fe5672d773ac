"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
published test vectors, closed forms, invariants stated by the paper, library special cases,
an independent float64 torch composition (forward) with autograd (adjoint), finite differences.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2605_02726_gb300 import inputs
from tests import torch_ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------------------------
# counter RNG
# ---------------------------------------------------------------------------------------------
def test_splitmix64_published_vectors():
    gamma = 0x9E3779B97F4A7C15
    for n, hexval in _read_golden("splitmix64.txt"):
        z = (int(n) * gamma) & ((1 << 64) - 1)
        assert oracle.splitmix64_mix(z) == int(hexval, 16)


def test_noise_matches_definition_and_is_uniform():
    seed, t = 1234567, 5
    u = oracle.noise(seed, t, 4000)
    ref = torch_ref.splitmix_noise(seed, t, 4000)
    np.testing.assert_array_equal(u, ref)
    assert u.min() >= -0.5 and u.max() < 0.5
    assert abs(u.mean()) < 0.02
    assert abs(u.var() - 1.0 / 12.0) < 0.01
    # different step -> different draw
    assert not np.array_equal(u[:100], oracle.noise(seed, t + 1, 100))


# ---------------------------------------------------------------------------------------------
# Laplace mass (Eq. 3)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("mu,b", [(0.0, 1.0), (0.3, 0.05), (-2.7, 7.0), (11.2, 0.7), (0.5, 0.01),
                                  (-0.49, 120.0)])
def test_laplace_mass_sums_to_one(mu, b):
    lo = math.floor(mu - 60 * b) - 2
    hi = math.ceil(mu + 60 * b) + 2
    tot = sum(oracle.laplace_prob(float(v), mu, b)[0] for v in range(lo, hi + 1))
    assert abs(tot - 1.0) < 1e-12


def test_laplace_closed_form_matches_cdf_difference_and_derivatives():
    rng = np.random.default_rng(0)
    for _ in range(300):
        mu = rng.uniform(-4, 4)
        b = math.exp(rng.uniform(-3, 3))
        y = rng.uniform(-6, 6)

        def cdf(z):
            return 0.5 + 0.5 * math.copysign(1.0, z) * (1 - math.exp(-abs(z) / b))

        direct = cdf(y + 0.5 - mu) - cdf(y - 0.5 - mu)
        p, dy, dlb = oracle.laplace_prob(y, mu, b)
        assert abs(p - direct) <= 1e-12 * max(1.0, direct) + 1e-15
        h = 1e-6
        fd_y = (oracle.laplace_prob(y + h, mu, b)[0] - oracle.laplace_prob(y - h, mu, b)[0]) / (2 * h)
        lb = math.log(b)
        fd_lb = (oracle.laplace_prob(y, mu, math.exp(lb + h))[0]
                 - oracle.laplace_prob(y, mu, math.exp(lb - h))[0]) / (2 * h)
        if abs(abs(y - mu) - 0.5) > 1e-4:  # the pdf is not differentiable at mu
            assert abs(fd_y - dy) < 1e-6 * max(1.0, abs(dy))
            assert abs(fd_lb - dlb) < 1e-6 * max(1.0, abs(dlb))


# ---------------------------------------------------------------------------------------------
# upsampling (Sec. III-B)
# ---------------------------------------------------------------------------------------------
def test_bicubic_taps_from_keys_kernel():
    rows = _read_golden("keys_bicubic.txt")
    a = -0.75

    def keys(x):
        x = abs(x)
        if x <= 1:
            return (a + 2) * x ** 3 - (a + 3) * x ** 2 + 1
        return a * x ** 3 - 5 * a * x ** 2 + 8 * a * x - 4 * a

    for dist, val in rows:
        assert keys(float(dist)) == float(val)
    assert tuple(float(v) for _, v in rows) == inputs.BICUBIC_TAPS
    assert sum(inputs.BICUBIC_TAPS) == 1.0


@pytest.mark.parametrize("shape,target", [((5, 7), (10, 14)), ((4, 6), (7, 11)), ((1, 1), (2, 1)),
                                          ((3, 2), (5, 4)), ((1, 3), (1, 6))])
def test_upsample_constant_stays_constant(shape, target):
    rng = np.random.default_rng(1)
    taps = rng.uniform(-0.3, 1.0, 4)
    taps = taps / taps.sum()
    out = oracle.upsample(np.full(shape, 2.5), taps, target)
    np.testing.assert_allclose(out, 2.5, rtol=0, atol=1e-14)


def test_upsample_delta_filter_is_nearest_neighbour():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(6, 9))
    out = oracle.upsample(x, [0.0, 0.0, 0.0, 1.0], (11, 18))
    ref = np.repeat(np.repeat(x, 2, axis=0), 2, axis=1)[:11, :18]
    np.testing.assert_array_equal(out, ref)


@pytest.mark.parametrize("shape,target", [((5, 7), (10, 14)), ((4, 6), (7, 11)), ((2, 3), (3, 5)),
                                          ((1, 1), (1, 2))])
def test_upsample_matches_transposed_conv(shape, target):
    rng = np.random.default_rng(3)
    x = rng.normal(size=shape)
    taps = rng.normal(size=4)
    out = oracle.upsample(x, taps, target)
    ref = torch_ref.upsample2d(torch.tensor(x)[None], torch.tensor(taps), *target)[0].numpy()
    np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------------------------------
# residual 3x3 conv and Adam: library special cases
# ---------------------------------------------------------------------------------------------
def test_conv3x3_residual_matches_torch_conv2d():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(3, 7, 5))
    w = rng.normal(size=(3, 3, 3, 3))
    b = rng.normal(size=3)
    out = oracle.conv3x3_res(x, w, b)
    xt = torch.tensor(x)[None]
    ref = xt[0] + torch.nn.functional.conv2d(
        torch.nn.functional.pad(xt, (1, 1, 1, 1), mode="replicate"), torch.tensor(w), torch.tensor(b))[0]
    np.testing.assert_allclose(out, ref.numpy(), rtol=1e-13, atol=1e-13)


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(5)
    p0 = rng.normal(size=50)
    p = p0.copy()
    m = np.zeros(50)
    v = np.zeros(50)
    pt = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 8):
        g = rng.normal(size=50)
        oracle.adam(p, g, m, v, step)
        opt.zero_grad()
        pt.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------------------------
# whole forward / adjoint against the independent torch composition
# ---------------------------------------------------------------------------------------------
SHAPES = [(8, 8), (13, 11), (16, 16), (24, 40)]


@pytest.mark.parametrize("H,W", SHAPES)
def test_forward_matches_torch_composition(H, W):
    img = inputs.image(H, W, seed=7).astype(np.float64)
    lat, par = inputs.random_state(H, W, seed=8)
    lat = lat.astype(np.float64)
    par = par.astype(np.float64)
    seed, step = 99, 3
    yt = lat + torch_ref.splitmix_noise(seed, step, lat.shape[0])
    o = oracle.forward(img, lat, par, lam=1e-2, seed=seed, step=step, per_latent=True)
    loss, rate, mse, mu, logb, xh = torch_ref.forward(torch.tensor(img), torch.tensor(yt), torch.tensor(par), 1e-2)
    assert abs(o["loss"] - loss.item()) <= 1e-12 * abs(loss.item())
    assert abs(o["rate_bits"] - rate.item()) <= 1e-11 * abs(rate.item())
    assert abs(o["mse"] - mse.item()) <= 1e-12 * abs(mse.item())
    np.testing.assert_allclose(o["mu"], mu.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(o["logb"], logb.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(o["xhat"], xh.numpy(), rtol=1e-12, atol=1e-12)
    # identity mode on pre-relaxed latents gives the same numbers
    o2 = oracle.forward(img, yt, par, lam=1e-2, mode=oracle.MODE_IDENTITY)
    assert abs(o2["loss"] - o["loss"]) <= 1e-14 * abs(o["loss"])


@pytest.mark.parametrize("H,W", SHAPES)
def test_adjoint_matches_torch_autograd(H, W):
    img = inputs.image(H, W, seed=17).astype(np.float64)
    lat, par = inputs.random_state(H, W, seed=18)
    yt = lat.astype(np.float64)
    par = par.astype(np.float64)
    o = oracle.loss_grad(img, yt, par, lam=3e-2, mode=oracle.MODE_IDENTITY)
    r = torch_ref.loss_and_grads(img, yt, par, 3e-2)
    assert abs(o["loss"] - r["loss"]) <= 1e-12 * abs(r["loss"])
    for key in ("grad_latents", "grad_params"):
        a, b = o[key], r[key]
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= 1e-10 * scale, key


def test_hard_quantisation_is_rint_and_has_no_latent_gradient():
    H, W = 16, 12
    img = inputs.image(H, W, seed=1).astype(np.float64)
    lat, par = inputs.random_state(H, W, seed=2)
    lat = lat.astype(np.float64)
    lat[:4] = [0.5, 1.5, -0.5, 2.5]  # ties round to even
    q = np.rint(lat)
    assert list(q[:4]) == [0.0, 2.0, -0.0, 2.0]
    a = oracle.forward(img, lat, par.astype(np.float64), lam=1e-3, mode=oracle.MODE_HARD)
    b = oracle.forward(img, q, par.astype(np.float64), lam=1e-3, mode=oracle.MODE_IDENTITY)
    assert a["loss"] == b["loss"]
    g = oracle.loss_grad(img, lat, par.astype(np.float64), lam=1e-3, mode=oracle.MODE_HARD)
    assert not np.any(g["grad_latents"])


# ---------------------------------------------------------------------------------------------
# finite differences (FP64, central) on tiny images
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("H,W", [(8, 8), (16, 16), (13, 9)])
def test_gradient_matches_central_differences(H, W):
    img = inputs.image(H, W, seed=21).astype(np.float64)
    lat, par = inputs.random_state(H, W, seed=22)
    yt = lat.astype(np.float64)
    par = par.astype(np.float64)
    lam = 2e-2
    g = oracle.loss_grad(img, yt, par, lam=lam, mode=oracle.MODE_IDENTITY)

    def f(y, p):
        return oracle.forward(img, y, p, lam=lam, mode=oracle.MODE_IDENTITY)["loss"]

    rng = np.random.default_rng(23)
    checked = 0
    coords = [("lat", i) for i in rng.choice(yt.shape[0], 40, replace=False)]
    coords += [("par", i) for i in rng.choice(par.shape[0], 60, replace=False)]
    for kind, i in coords:
        def fd(h):
            y2, p2 = yt.copy(), par.copy()
            arr = y2 if kind == "lat" else p2
            arr[i] += h
            fp = f(y2, p2)
            arr[i] -= 2 * h
            fm = f(y2, p2)
            return (fp - fm) / (2 * h)

        d1, d2 = fd(1e-4), fd(5e-5)
        an = (g["grad_latents"] if kind == "lat" else g["grad_params"])[i]
        scale = max(abs(an), 1e-7)
        if abs(d1 - d2) > 1e-6 * scale:  # a ReLU kink or clamp edge inside +-h: skip
            continue
        checked += 1
        assert abs(d1 - an) <= 1e-5 * scale + 1e-11, (kind, i, d1, an)
    assert checked >= 80


# ---------------------------------------------------------------------------------------------
# causality of the entropy model (Eq. 2 conditions on already decoded values only)
# ---------------------------------------------------------------------------------------------
def test_arm_is_causal_and_ifce_reads_only_coarser_grids():
    H, W = 16, 24
    img = inputs.image(H, W, seed=31).astype(np.float64)
    lat, par = inputs.random_state(H, W, seed=32)
    y = lat.astype(np.float64)
    par = par.astype(np.float64)
    shapes = inputs.grid_shapes(H, W)
    offs = np.cumsum([0] + [h * w for h, w in shapes])
    base = oracle.forward(img, y, par, lam=1e-2, mode=oracle.MODE_IDENTITY, per_latent=True)
    rng = np.random.default_rng(33)
    for k in range(7):
        h, w = shapes[k]
        for _ in range(3):
            r, c = int(rng.integers(h)), int(rng.integers(w))
            j = offs[k] + r * w + c
            y2 = y.copy()
            y2[j] += 3.7
            o = oracle.forward(img, y2, par, lam=1e-2, mode=oracle.MODE_IDENTITY, per_latent=True)
            # same grid: every position at or before (r, c) in raster order is unchanged
            before = np.arange(offs[k], j + 1)
            np.testing.assert_array_equal(o["mu"][before], base["mu"][before])
            np.testing.assert_array_equal(o["logb"][before], base["logb"][before])
            # coarser grids are decoded earlier: unchanged
            np.testing.assert_array_equal(o["mu"][offs[k + 1]:], base["mu"][offs[k + 1]:])
            # finer grids without an IFCE (k' >= 3) never read grid k
            for kk in range(3, k):
                sl = slice(offs[kk], offs[kk + 1])
                np.testing.assert_array_equal(o["mu"][sl], base["mu"][sl])
            # some later position of the same grid does change (the context is live)
            if r * w + c < h * w - 1 and (c > 0 or r + 1 < h):
                after = np.arange(j + 1, offs[k + 1])
                assert np.any(o["mu"][after] != base["mu"][after]) or h * w < 4


# ---------------------------------------------------------------------------------------------
# integer decode CDF
# ---------------------------------------------------------------------------------------------
def test_cdf_tables_closed_forms():
    # K[0] = rint(2^20 log2 e) = rint(1512775.395...)
    assert oracle.table_entry(0, 1280) == 1512775
    assert oracle.table_entry(1, 0) == 32768 and oracle.table_entry(2, 0) == 32768
    # T_HI[512] = rint(2^15 / sqrt 2) = rint(23170.475...)
    assert oracle.table_entry(1, 512) == 23170


@pytest.mark.parametrize("s,mu_q", [(0, 0), (-1280, 37), (1280, -500), (-600, 128), (300, 77), (-1000, -3)])
def test_integer_cdf_telescopes_and_tracks_laplace(s, mu_q):
    b = math.exp(s / 256.0)
    span = int(60 * b) + 4
    tot = 0
    for v in range(-span, span + 1):
        tp = 256 * v + 128 - mu_q
        tm = 256 * v - 128 - mu_q
        tot += oracle.cdf_q16(s, tp) - oracle.cdf_q16(s, tm)
    assert tot == 65536
    # C(t)/65536 within a few 2^-16 of the exact Laplace CDF at z = t/256
    for t in list(range(-3000, 3001, 37)) + [0, 1, -1, 255, -255]:
        z = t / 256.0
        exact = 0.5 + 0.5 * math.copysign(1.0, z) * (1 - math.exp(-abs(z) / b)) if z != 0 else 0.5
        assert abs(oracle.cdf_q16(s, t) / 65536.0 - exact) <= 4.0 / 65536.0
    # monotone in t
    prev = -1
    for t in range(-5000, 5000, 13):
        c = oracle.cdf_q16(s, t)
        assert c >= prev
        prev = c


def test_decode_probabilities_are_valid():
    H, W = 16, 16
    q = inputs.quantized_latents(H, W, seed=41)
    _, par = inputs.random_state(H, W, seed=42)
    d = oracle.decode_probs(H, W, q, par)
    assert d["prob_q16"].min() >= 1 and d["prob_q16"].max() <= 65536
    assert d["logb_q"].min() >= -1280 and d["logb_q"].max() <= 1280
    # fixed point tracks the float ARM of the unquantised weights
    fl = oracle.forward(np.zeros((3, H, W)), q.astype(np.float64), par.astype(np.float64), lam=0.0,
                        mode=oracle.MODE_IDENTITY, per_latent=True)
    assert np.abs(d["mu_q"] / 256.0 - fl["mu"]).max() < 0.25


def _q8(par):
    """Parameters on the decoder's 2^-8 grid, as FP64 values."""
    return np.rint(par.astype(np.float64) * 256.0) / 256.0


def test_decode_fixed_point_arm_within_its_floor_bound():
    """The integer ARM computes the FP64 ARM of the same integer latents and of the weights
    rounded to the 2^-8 grid, except that each hidden or output layer floors its result to the
    2^-8 grid.  A floor lowers a value by less than 2^-8, ReLU does not enlarge a difference, and
    a layer scales the difference it receives by the l1 norm of its weight rows, so
        e1 = 2^-8,  e2[o] = 2^-8 + sum_n |W2[o,n]| e1,  e_out[o] = 2^-8 + sum_n |W3[o,n]| e2[n]
    bounds |mu_q / 256 - mu| and |logb_q / 256 - log b| (the clamp to [-5, 5] is 1-Lipschitz).  The
    IFCE and the spatial context enter the integer ARM exactly (products of integers)."""
    H, W = 24, 40
    q = inputs.quantized_latents(H, W, seed=41)
    _, par = inputs.random_state(H, W, seed=42)
    d = oracle.decode_probs(H, W, q, par)
    pq = _q8(par)
    fl = oracle.forward(np.zeros((3, H, W)), q.astype(np.float64), pq, lam=0.0, mode=oracle.MODE_IDENTITY,
                        per_latent=True)
    W2 = torch_ref.P(torch.tensor(pq), "arm.w2").numpy()
    W3 = torch_ref.P(torch.tensor(pq), "arm.w3").numpy()
    u = 2.0 ** -8
    e2 = u + np.abs(W2) @ np.full(16, u)
    e_out = u + np.abs(W3) @ e2
    assert np.abs(d["mu_q"] / 256.0 - fl["mu"]).max() <= e_out[0] + 1e-12
    assert np.abs(d["logb_q"] / 256.0 - fl["logb"]).max() <= e_out[1] + 1e-12
    # the bound is not vacuous: it is far below the size of the biases it would have to hide
    assert e_out.max() < 0.05
    # every latent of grids 0..2 went through its IFCE: the IFCE weights matter
    assert np.any(np.abs(torch_ref.P(torch.tensor(pq), "ifce0.w").numpy()) > 0)


def test_decode_probability_is_the_laplace_mass_of_its_integer_parameters():
    """P_q16 = max(1, C(t+) - C(t-)) with C/65536 within 4 * 2^-16 of the Laplace CDF (pinned above), so
    P_q16 is within 8 of 65536 times the exact mass of [y - 1/2, y + 1/2) under the Laplace law of
    mean mu_q / 256 and scale exp(logb_q / 256) (Eq. 3); the floor at 1 stays inside that bound."""
    H, W = 24, 40
    q = inputs.quantized_latents(H, W, seed=43)
    _, par = inputs.random_state(H, W, seed=44)
    d = oracle.decode_probs(H, W, q, par)
    mu = d["mu_q"].astype(np.float64) / 256.0
    b = np.exp(d["logb_q"].astype(np.float64) / 256.0)

    def cdf(z):
        return 0.5 + 0.5 * np.sign(z) * (1.0 - np.exp(-np.abs(z) / b))

    mass = cdf(q + 0.5 - mu) - cdf(q - 0.5 - mu)
    assert np.abs(d["prob_q16"].astype(np.float64) - 65536.0 * mass).max() <= 8.0
    # both tails and the centre are exercised
    assert (mass < 1e-4).any() and (mass > 0.5).any()


def test_encode_iteration_is_loss_grad_then_adam():
    """One iteration of the uniform-proxy encoder from step t: the loss and gradient with the noise
    keyed by t, then Adam with step count t + 1 on latents and parameters (Sec. IV-B), then the
    next iteration keyed by t + 1."""
    H, W = 8, 12
    img = inputs.image(H, W, seed=12)
    lat, par = inputs.random_state(H, W, seed=13)
    lam, seed, t0 = 1e-2, 77, 3
    st = oracle.State(lat, par, step=t0)
    out = oracle.encode(img, st, 2, lam=lam, seed=seed)
    assert st.step == t0 + 2

    ref = oracle.State(lat, par, step=t0)
    for it in range(2):
        g = oracle.loss_grad(img, ref.latents, ref.params, lam=lam, mode=oracle.MODE_NOISE, seed=seed,
                             step=t0 + it)
        assert abs(g["loss"] - out["loss"][it]) <= 1e-15 * abs(g["loss"])
        assert abs(g["rate_bits"] - out["rate_bits"][it]) <= 1e-15 * abs(g["rate_bits"])
        oracle.adam(ref.latents, g["grad_latents"], ref.m_lat, ref.v_lat, t0 + it + 1, lr=1e-2)
        oracle.adam(ref.params, g["grad_params"], ref.m_par, ref.v_par, t0 + it + 1, lr=1e-2)
    np.testing.assert_allclose(st.latents, ref.latents, rtol=0, atol=1e-15)
    np.testing.assert_allclose(st.params, ref.params, rtol=0, atol=1e-15)
    np.testing.assert_allclose(st.m_lat, ref.m_lat, rtol=0, atol=1e-15)
    np.testing.assert_allclose(st.v_par, ref.v_par, rtol=0, atol=1e-15)
    # a slip of the noise key would show: the neighbouring key gives another loss
    other = oracle.forward(img, lat, par, lam=lam, mode=oracle.MODE_NOISE, seed=seed, step=t0 + 1)
    assert abs(other["loss"] - out["loss"][0]) > 1e-9 * abs(out["loss"][0])
    # a slip of the Adam count would show: bias correction at t0 + 2 instead of t0 + 1
    slip = oracle.State(lat, par, step=t0)
    g = oracle.loss_grad(img, slip.latents, slip.params, lam=lam, mode=oracle.MODE_NOISE, seed=seed, step=t0)
    one = oracle.State(lat, par, step=t0)
    oracle.encode(img, one, 1, lam=lam, seed=seed)
    oracle.adam(slip.latents, g["grad_latents"], slip.m_lat, slip.v_lat, t0 + 2, lr=1e-2)
    assert np.abs(slip.latents - one.latents).max() > 1e-6
