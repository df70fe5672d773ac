"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module only draws random numbers: images shaped like the paper's test sets (Kodak
512x768, CLIC20 384x512..1370x2048 -- neither dataset is available here, so 1/f^2 Gaussian
fields stand in for them) and initial encoder states.  It holds none of the method's
arithmetic, so both the CUDA path and the FP64 oracle may consume what it produces.

The flat parameter layout below is the interface of the C library (``include/coolchic.h``);
it is restated here only to know which block gets which initialisation.
"""
from __future__ import annotations

import numpy as np

SEED0 = 20260
N_GRIDS = 7

# (name, shape) of every parameter block, in storage order (row-major [out][in]).
PARAM_BLOCKS = [
    ("arm.w1", (16, 20)), ("arm.b1", (16,)), ("arm.w2", (16, 16)), ("arm.b2", (16,)),
    ("arm.w3", (2, 16)), ("arm.b3", (2,)), ("arm.ws", (2, 20)), ("arm.bs", (2,)),
    ("ifce0.w", (4, 6)), ("ifce0.b", (4,)), ("ifce1.w", (4, 5)), ("ifce1.b", (4,)),
    ("ifce2.w", (4, 4)), ("ifce2.b", (4,)),
    ("up.taps", (6, 4)),
    ("syn.w1", (40, 7)), ("syn.b1", (40,)), ("syn.w2", (3, 40)), ("syn.b2", (3,)),
    ("syn.ws", (3, 7)), ("syn.bs", (3,)),
    ("conv1.w", (3, 3, 3, 3)), ("conv1.b", (3,)), ("conv2.w", (3, 3, 3, 3)), ("conv2.b", (3,)),
]


def param_offsets():
    offs, o = {}, 0
    for name, shape in PARAM_BLOCKS:
        n = int(np.prod(shape))
        offs[name] = (o, shape)
        o += n
    return offs, o


PARAM_OFFSETS, N_PARAMS = param_offsets()
assert N_PARAMS == 1415

# Hyperlatent grids (optional, Sec. III-A3): three more grids at 1/16, 1/32, 1/64 of the image whose
# latents follow the main ones; the IFCE weights of their inputs follow the 1415 main parameters as
# one block [grid k = 0..2][output o = 0..3][hyperlatent grid q = 0..2].
N_HYPER_GRIDS = 3
HYPER_BLOCK = ("ifce_h.w", (3, 4, 3))
N_PARAMS_H = N_PARAMS + 36

# Keys cubic kernel (a = -0.75) sampled at distances 1.75, 1.25, 0.75, 0.25: exact binary fractions.
BICUBIC_TAPS = (-0.03515625, -0.10546875, 0.26171875, 0.87890625)


def grid_shapes(H: int, W: int, L: int = N_GRIDS, hyper: bool = False):
    """Latent grid shapes; with hyper, then the hyperlatent grids (shapes of grids 4, 5, 6)."""
    main = [(-(-H // (1 << k)), -(-W // (1 << k))) for k in range(L)]
    return main + ([(-(-H // (1 << k)), -(-W // (1 << k))) for k in range(4, 4 + N_HYPER_GRIDS)] if hyper else [])


def latent_count(H: int, W: int, hyper: bool = False) -> int:
    return sum(h * w for h, w in grid_shapes(H, W, hyper=hyper))


def block(params: np.ndarray, name: str) -> np.ndarray:
    o, shape = PARAM_OFFSETS[name]
    return params[o:o + int(np.prod(shape))].reshape(shape)


def image(H: int, W: int, seed: int, texture_sigma: float = 0.0) -> np.ndarray:
    """RGB image [3, H, W] float32 in [0, 1]: per channel a Gaussian field with amplitude
    spectrum 1/|f| (power 1/f^2, DC removed), min-max scaled; optional N(0, sigma^2) texture
    noise, clipped."""
    rng = np.random.default_rng(seed)
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    f = np.sqrt(fy * fy + fx * fx)
    f[0, 0] = 1.0
    out = np.empty((3, H, W), dtype=np.float64)
    for c in range(3):
        spec = (rng.standard_normal(f.shape) + 1j * rng.standard_normal(f.shape)) / f
        spec[0, 0] = 0.0
        field = np.fft.irfft2(spec, s=(H, W))
        lo, hi = field.min(), field.max()
        field = (field - lo) / (hi - lo) if hi > lo else np.zeros_like(field)
        if texture_sigma > 0.0:
            field = np.clip(field + rng.normal(0.0, texture_sigma, field.shape), 0.0, 1.0)
        out[c] = field
    return out.astype(np.float32)


def initial_state(H: int, W: int, seed: int, hyper: bool = False):
    """Encoder starting point: latents N(0, 0.01^2); hidden-layer weights U(+-1/sqrt(fan_in));
    biases, last layers, stabilizers and residual convs zero; upsampling taps bicubic.  With
    hyper, the hyperlatents and the IFCE weights of their inputs are drawn the same way (an IFCE's
    fan-in then counts its hyperlatent inputs too).
    Returns (latents float32 [N], params float32 [1415, or 1451 with hyper])."""
    rng = np.random.default_rng(seed)
    lat = rng.normal(0.0, 0.01, latent_count(H, W)).astype(np.float32)
    p = np.zeros(N_PARAMS, dtype=np.float64)
    for name in ("arm.w1", "arm.w2", "ifce0.w", "ifce1.w", "ifce2.w", "syn.w1"):
        o, shape = PARAM_OFFSETS[name]
        n = int(np.prod(shape))
        fan = shape[1] + (N_HYPER_GRIDS if hyper and name.startswith("ifce") else 0)
        bound = 1.0 / np.sqrt(fan)
        p[o:o + n] = rng.uniform(-bound, bound, n)
    block(p, "up.taps")[:] = BICUBIC_TAPS
    if hyper:
        lat = np.concatenate([lat, rng.normal(0.0, 0.01, latent_count(H, W, True) - lat.shape[0]).astype(np.float32)])
        fans = np.repeat([6 + 3, 5 + 3, 4 + 3], 12)
        p = np.concatenate([p, rng.uniform(-1.0, 1.0, 36) / np.sqrt(fans)])
    return lat, p.astype(np.float32)


def random_state(H: int, W: int, seed: int, latent_sigma: float = 1.5, scale: float = 1.0, hyper: bool = False):
    """A mid-training-like state for parity tests: every block random and non-zero so that
    every gradient path is exercised.  Returns (latents float32, params float32); with hyper the
    hyperlatents and their IFCE weights are appended (drawn after the main state, which is
    therefore the same with and without them)."""
    rng = np.random.default_rng(seed)
    lat = rng.normal(0.0, latent_sigma, latent_count(H, W)).astype(np.float32)
    p = np.zeros(N_PARAMS, dtype=np.float64)
    for name, shape in PARAM_BLOCKS:
        o, _ = PARAM_OFFSETS[name]
        n = int(np.prod(shape))
        if name == "up.taps":
            p[o:o + n] = np.tile(BICUBIC_TAPS, 6) + rng.uniform(-0.02, 0.02, n)
        elif name.startswith("conv") and name.endswith(".w"):
            p[o:o + n] = rng.uniform(-0.1, 0.1, n) * scale
        elif len(shape) == 1:
            p[o:o + n] = rng.uniform(-0.1, 0.1, n) * scale
        else:
            bound = 1.0 / np.sqrt(shape[1])
            p[o:o + n] = rng.uniform(-bound, bound, n) * scale
    # keep the Laplace log-scale away from its clamp and the mean near the latents
    block(p, "arm.b3")[:] = (0.0, 0.3)
    if hyper:
        lat = np.concatenate([lat, rng.normal(0.0, latent_sigma, latent_count(H, W, True) - lat.shape[0])
                              .astype(np.float32)])
        p = np.concatenate([p, rng.uniform(-0.4, 0.4, 36) * scale])
    return lat, p.astype(np.float32)


def quantized_latents(H: int, W: int, seed: int, sigma: float = 3.0, hyper: bool = False) -> np.ndarray:
    """Integer latents for decode tests (int32), Laplace-like spread."""
    rng = np.random.default_rng(seed)
    return np.rint(rng.laplace(0.0, sigma, latent_count(H, W, hyper))).astype(np.int32)


BATCH_SIZES = [(256, 256), (512, 768), (768, 512), (1024, 1024), (1536, 1024)]


def batch_workload(n_images: int = 32, seed0: int = SEED0):
    """Image sizes for the mixed-size batched encode: uniform over BATCH_SIZES."""
    rng = np.random.default_rng(seed0 - 1)
    idx = rng.integers(0, len(BATCH_SIZES), n_images)
    return [BATCH_SIZES[i] for i in idx]


SERVE_SIZES = [(512, 768), (1024, 1024), (2048, 1365), (2048, 2048)]
SERVE_WEIGHTS = [0.4, 0.3, 0.2, 0.1]
SERVE_LAMBDAS = [1e-4, 1e-3, 1e-2]


def serve_requests(rate_per_s: float, n_requests: int, seed0: int = SEED0):
    """Poisson arrivals: list of (arrival_time_s, (H, W), lambda)."""
    rng = np.random.default_rng(seed0 - 2 + int(rate_per_s * 1000))
    gaps = rng.exponential(1.0 / rate_per_s, n_requests)
    times = np.cumsum(gaps) - gaps[0]
    sizes = rng.choice(len(SERVE_SIZES), n_requests, p=SERVE_WEIGHTS)
    lams = rng.choice(SERVE_LAMBDAS, n_requests)
    return [(float(t), SERVE_SIZES[s], float(l)) for t, s, l in zip(times, sizes, lams)]
