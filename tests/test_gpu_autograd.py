"""Differentiation check on a 256x256 image: the hand-written adjoint behind torch.autograd.Function
(`paper_2605_02726_gb300.autograd.rd_loss`) against

  * central finite differences of the FP64 oracle loss (step 1e-3) on 200 seed-chosen coordinates,
    100 parameters and 100 latents, and
  * the oracle's full FP64 gradient (1e-3 of each block's largest magnitude),

with the activations recomputed per tile (recompute=True) and stored by the forward
(recompute=False).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_02726_gb300 import inputs

pytestmark = pytest.mark.gpu

H = W = 256
LAM = 1e-2
SEED = 77
STEP = 3
FD_STEP = 1e-3
N_PARAM_COORDS = N_LATENT_COORDS = 100


@pytest.fixture(scope="module")
def problem():
    img = inputs.image(H, W, seed=901)
    lat, par = inputs.random_state(H, W, seed=902)
    o = oracle.loss_grad(img, lat, par, lam=LAM, mode=oracle.MODE_NOISE, seed=SEED, step=STEP)
    return img, lat, par, o


def _gpu(cc, img, lat, par, recompute, outer=1.0):
    from paper_2605_02726_gb300.autograd import rd_loss
    gi = torch.tensor(img, device="cuda")
    gl = torch.tensor(lat, device="cuda", requires_grad=True)
    gp = torch.tensor(par, device="cuda", requires_grad=True)
    loss, rate, mse = rd_loss(gl, gp, gi, H=H, W=W, hp=cc.hparams(lam=LAM, seed=SEED), step=STEP,
                              recompute=recompute)
    (loss * outer).backward()
    assert not rate.requires_grad and not mse.requires_grad
    return float(loss.detach()), gl.grad.double().cpu().numpy(), gp.grad.double().cpu().numpy()


@pytest.fixture(scope="module")
def gpu_grads(cc, problem):
    img, lat, par, _ = problem
    return {rc: _gpu(cc, img, lat, par, rc) for rc in (True, False)}


def _blocks():
    """(name, slice into latents or params, is_latent)"""
    out, off = [], 0
    for k, (h, w) in enumerate(inputs.grid_shapes(H, W)):
        out.append((f"latents grid {k}", slice(off, off + h * w), True))
        off += h * w
    for name, (po, shape) in inputs.PARAM_OFFSETS.items():
        out.append((name, slice(po, po + int(np.prod(shape))), False))
    return out


def _block_max(o):
    """largest oracle-gradient magnitude of the block each coordinate belongs to"""
    lat_max = np.zeros_like(o["grad_latents"])
    par_max = np.zeros_like(o["grad_params"])
    for _, sl, is_lat in _blocks():
        src, dst = (o["grad_latents"], lat_max) if is_lat else (o["grad_params"], par_max)
        dst[sl] = np.abs(src[sl]).max()
    return lat_max, par_max


@pytest.mark.parametrize("recompute", [True, False])
def test_autograd_matches_oracle_gradient(problem, gpu_grads, recompute):
    _, _, _, o = problem
    loss, gl, gp = gpu_grads[recompute]
    assert abs(loss - o["loss"]) <= 1e-4 * abs(o["loss"])
    for name, sl, is_lat in _blocks():
        g, ref = (gl, o["grad_latents"]) if is_lat else (gp, o["grad_params"])
        scale = np.abs(ref[sl]).max()
        err = np.abs(g[sl] - ref[sl]).max()
        assert err <= 1e-3 * scale + 1e-30, f"{name}: max err {err:.3e}, block max {scale:.3e}"


def test_recompute_and_stored_agree(gpu_grads):
    l1, gl1, gp1 = gpu_grads[True]
    l0, gl0, gp0 = gpu_grads[False]
    assert l1 == l0
    for a, b in ((gl1, gl0), (gp1, gp0)):
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()


def test_outer_gradient_scales(cc, problem, gpu_grads):
    img, lat, par, _ = problem
    _, gl3, gp3 = _gpu(cc, img, lat, par, True, outer=3.0)
    _, gl1, gp1 = gpu_grads[True]
    np.testing.assert_allclose(gl3, 3.0 * gl1, rtol=1e-6, atol=1e-6 * np.abs(gl1).max())
    np.testing.assert_allclose(gp3, 3.0 * gp1, rtol=1e-6, atol=1e-6 * np.abs(gp1).max())


def test_autograd_matches_finite_differences(problem, gpu_grads):
    """Central differences of the FP64 oracle loss; coordinates where the one-sided differences
    disagree (a ReLU kink or a clamp inside the step) are skipped, at most 10% of them."""
    img, lat, par, o = problem
    rng = np.random.default_rng(4242)
    coords = [("p", int(j)) for j in rng.choice(oracle.N_PARAMS, N_PARAM_COORDS, replace=False)]
    coords += [("y", int(j)) for j in rng.choice(lat.shape[0], N_LATENT_COORDS, replace=False)]
    lat64, par64 = lat.astype(np.float64), par.astype(np.float64)

    def loss_at(kind, j, dx):
        la, pa = lat64, par64
        if kind == "y":
            la = lat64.copy()
            la[j] += dx
        else:
            pa = par64.copy()
            pa[j] += dx
        return oracle.forward(img, la, pa, lam=LAM, mode=oracle.MODE_NOISE, seed=SEED, step=STEP)["loss"]

    lat_max, par_max = _block_max(o)
    l0 = o["loss"]
    checked, bad = 0, []
    for kind, j in coords:
        lp, lm = loss_at(kind, j, FD_STEP), loss_at(kind, j, -FD_STEP)
        fd = (lp - lm) / (2 * FD_STEP)
        fwd, bwd = (lp - l0) / FD_STEP, (l0 - lm) / FD_STEP
        scale = lat_max[j] if kind == "y" else par_max[j]
        if abs(fwd - bwd) > 1e-2 * (abs(fd) + scale):
            continue  # non-smooth inside the step
        checked += 1
        for recompute in (True, False):
            _, gl, gp = gpu_grads[recompute]
            g = gl[j] if kind == "y" else gp[j]
            if abs(g - fd) > 1e-3 * scale + 1e-3 * abs(fd):
                bad.append((kind, j, recompute, g, fd, scale))
    assert checked >= 0.9 * len(coords), f"only {checked} of {len(coords)} coordinates are smooth at this step"
    assert not bad, f"{len(bad)} mismatches, first: {bad[:3]}"
