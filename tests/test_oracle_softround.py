"""Pins of the oracle's soft-round proxy (Eq. 13-14) and encoder schedule (Sec. IV-C/D, Table I).

Checked against properties the paper and the mathematics fix, not against the oracle itself:
soft rounding is exact at the integers, continuous and continuously differentiable across them,
odd about the half-integers, tends to the identity for large T and to rint for small T; its
derivative matches finite differences; the Gaussian draws are the Box-Muller transform of the
counter hash (restated here from the published method) with the moments of N(0, 1); the latent
gradient through the proxy matches finite differences of the loss; the schedule freezes the
latents in the hard-round stage and follows its formulas in the main stage.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_02726_gb300 import inputs


@pytest.mark.parametrize("T", [0.08, 0.2, 0.35, 1.0])
def test_softround_integers_continuity_symmetry(T):
    for n in range(-5, 6):
        v, _ = oracle.softround(float(n), T)
        assert v == float(n)
        left, dl = oracle.softround(n - 1e-12, T)
        right, dr = oracle.softround(n + 1e-12, T)
        assert abs(left - n) < 1e-10 and abs(right - n) < 1e-10
        assert abs(dl - dr) < 1e-6 * max(1.0, dl)  # C1 across the integer
        for d in (0.1, 0.23, 0.4):
            up, _ = oracle.softround(n + 0.5 + d, T)
            dn, _ = oracle.softround(n + 0.5 - d, T)
            assert abs((up - (n + 0.5)) + (dn - (n + 0.5))) < 1e-12  # odd about n + 1/2


def test_softround_limits():
    xs = np.linspace(-3.3, 3.7, 71)
    for x in xs:
        assert abs(oracle.softround(float(x), 1e3)[0] - x) < 1e-6  # T -> inf: identity
        if abs(x - math.floor(x) - 0.5) > 0.05:
            assert abs(oracle.softround(float(x), 0.005)[0] - round(x)) < 1e-6  # T -> 0: rounding


@pytest.mark.parametrize("T", [0.08, 0.35])
def test_softround_derivative_matches_finite_differences(T):
    h = 1e-6
    for x in np.linspace(-2.4, 2.6, 23):
        _, d = oracle.softround(float(x), T)
        fd = (oracle.softround(x + h, T)[0] - oracle.softround(x - h, T)[0]) / (2 * h)
        assert abs(d - fd) < 1e-5 * max(1.0, abs(d))


def _box_muller_reference(seed, t, n):
    """SplitMix64 of seed ^ ((t << 32) + i) * gamma; u1 = (bits 40..63 + 1/2) / 2^24,
    u2 = bits 16..39 / 2^24; n = sqrt(-2 ln u1) cos(2 pi u2) (Box and Muller, 1958)."""
    M = (1 << 64) - 1
    out = np.empty(n)
    for i in range(n):
        z = (seed ^ ((((t << 32) + i) * 0x9E3779B97F4A7C15) & M)) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        z ^= z >> 31
        u1 = ((z >> 40) + 0.5) / 16777216.0
        u2 = ((z >> 16) & 0xFFFFFF) / 16777216.0
        out[i] = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
    return out


def test_gauss_is_box_muller_of_the_counter_hash():
    g = oracle.gauss(99, 7, 3000)
    np.testing.assert_allclose(g, _box_muller_reference(99, 7, 3000), rtol=0, atol=1e-12)


def test_gauss_moments():
    n = 200_000
    g = oracle.gauss(2026, 3, n)
    se = 1.0 / math.sqrt(n)
    assert abs(g.mean()) < 5 * se
    assert abs(g.var() - 1.0) < 5 * math.sqrt(2.0) * se
    assert abs(np.mean(g ** 3)) < 5 * math.sqrt(15.0) * se
    assert abs(np.mean(g ** 4) - 3.0) < 5 * math.sqrt(96.0) * se
    assert not np.array_equal(g[:50], oracle.gauss(2026, 4, 50))


def test_softround_proxy_reduces_to_rounding():
    """sigma = 0 and a tiny temperature: the proxy (Eq. 13) is the hard rounding of Eq. 12."""
    H, W = 12, 10
    img = inputs.image(H, W, seed=4)
    lat, par = inputs.random_state(H, W, seed=5, latent_sigma=1.3)
    lat = lat.astype(np.float64)
    frac = lat - np.floor(lat)
    lat[np.abs(frac - 0.5) < 0.02] += 0.05  # keep away from the rounding ties
    a = oracle.forward(img, lat, par, lam=1e-2, mode=oracle.MODE_SOFTROUND, sigma=0.0, temp=1e-3)
    b = oracle.forward(img, lat, par, lam=1e-2, mode=oracle.MODE_HARD)
    assert abs(a["loss"] - b["loss"]) < 1e-9 * abs(b["loss"])


def test_latent_gradient_through_the_proxy_matches_finite_differences():
    H, W = 10, 9
    img = inputs.image(H, W, seed=6)
    lat, par = inputs.random_state(H, W, seed=7, latent_sigma=1.0)
    lat = lat.astype(np.float64)
    kw = dict(lam=2e-2, mode=oracle.MODE_SOFTROUND, seed=3, step=11, sigma=0.2, temp=0.3)
    g = oracle.loss_grad(img, lat, par, **kw)["grad_latents"]
    rng = np.random.default_rng(8)
    h = 1e-5
    checked = 0
    for i in rng.choice(lat.shape[0], 25, replace=False):
        lp, lm = lat.copy(), lat.copy()
        lp[i] += h
        lm[i] -= h
        fp, fm, f0 = (oracle.forward(img, x, par, **kw)["loss"] for x in (lp, lm, lat))
        fd = (fp - fm) / (2 * h)
        if abs((fp - f0) - (f0 - fm)) > 1e-3 * abs(fp - fm) + 1e-12:
            continue  # a ReLU kink or clamp inside the step
        checked += 1
        assert abs(g[i] - fd) <= 1e-5 * max(abs(fd), np.abs(g).max())
    assert checked >= 20


def test_schedule_main_stage_then_frozen_latents():
    H, W = 8, 8
    img = inputs.image(H, W, seed=9)
    lat, par = inputs.initial_state(H, W, seed=10)
    lam, seed, n_main = 1e-2, 5, 3
    st = oracle.State(lat, par)
    out = oracle.encode_schedule(img, st, 5, lam=lam, seed=seed, n_main=n_main)
    assert st.step == 5 and np.all(np.isfinite(out["loss"]))

    # the first main-stage iteration equals its formulas: proxy at (sigma0, T0), Adam at lr_max
    ref = oracle.State(lat, par)
    g = oracle.loss_grad(img, ref.latents, ref.params, lam=lam, mode=oracle.MODE_SOFTROUND, seed=seed,
                         step=0, sigma=0.22, temp=0.35)
    assert abs(g["loss"] - out["loss"][0]) < 1e-12 * abs(g["loss"])
    ref.step = 0
    one = oracle.State(lat, par)
    oracle.encode_schedule(img, one, 1, lam=lam, seed=seed, n_main=n_main)
    oracle.adam(ref.latents, g["grad_latents"], ref.m_lat, ref.v_lat, 1, lr=1e-2)
    oracle.adam(ref.params, g["grad_params"], ref.m_par, ref.v_par, 1, lr=1e-2)
    np.testing.assert_allclose(one.latents, ref.latents, rtol=0, atol=1e-15)
    np.testing.assert_allclose(one.params, ref.params, rtol=0, atol=1e-15)

    # hard-round stage (steps 3, 4): latents and their moments frozen, loss of the rounded latents
    mid = oracle.State(lat, par)
    oracle.encode_schedule(img, mid, n_main, lam=lam, seed=seed, n_main=n_main)
    y_before, m_before = mid.latents.copy(), mid.m_lat.copy()
    p_before = mid.params.copy()
    hard = oracle.encode_schedule(img, mid, 2, lam=lam, seed=seed, n_main=n_main)
    np.testing.assert_array_equal(mid.latents, y_before)
    np.testing.assert_array_equal(mid.m_lat, m_before)
    assert not np.array_equal(mid.params, p_before)
    h0 = oracle.forward(img, y_before, p_before, lam=lam, mode=oracle.MODE_HARD)
    assert abs(hard["loss"][0] - h0["loss"]) < 1e-12 * abs(h0["loss"])
