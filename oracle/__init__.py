"""FP64 CPU oracle of the Cool-chic 5.0 encoder step -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The product path (``paper_2605_02726_gb300``) never imports it and shares no code
with it: the oracle is plain C (``coolchic_oracle.c``) compiled with gcc, loaded here through
ctypes, with numpy float64 arrays as arguments.

Every function follows a passage of the paper; see the header of ``coolchic_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "coolchic_oracle.c")
_SO = os.path.join(_HERE, "_coolchic_oracle.so")
_lock = threading.Lock()
_lib = None

N_GRIDS = 7
N_PARAMS = 1415
N_HYPER_GRIDS = 3
N_PARAMS_H = N_PARAMS + 3 * 4 * N_HYPER_GRIDS  # + IFCE weights of the hyperlatent inputs
MODE_NOISE, MODE_HARD, MODE_IDENTITY, MODE_SOFTROUND = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle into a shared object next to its source (gcc, OpenMP, no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        I32 = ctypes.POINTER(ctypes.c_int32)
        U32 = ctypes.POINTER(ctypes.c_uint32)
        F32 = ctypes.POINTER(ctypes.c_float)
        i64 = ctypes.c_int64
        u64 = ctypes.c_uint64
        c_int = ctypes.c_int
        dbl = ctypes.c_double
        sig = {
            "orc_param_count": (c_int, [c_int]),
            "orc_latent_count": (i64, [c_int, c_int, c_int]),
            "orc_grid_shape": (None, [c_int, c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
            "orc_context_offsets": (None, [ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
            "orc_splitmix64_mix": (u64, [u64]),
            "orc_noise": (dbl, [u64, i64, i64]),
            "orc_gauss": (dbl, [u64, i64, i64]),
            "orc_softround": (dbl, [dbl, dbl, D]),
            "orc_laplace_prob": (dbl, [dbl, dbl, dbl, D, D]),
            "orc_upsample": (None, [c_int, c_int, c_int, c_int, D, D, D]),
            "orc_conv3x3_res": (None, [c_int, c_int, D, D, D, D]),
            "orc_forward": (dbl, [c_int, c_int, c_int, D, D, D, c_int, u64, i64, dbl, dbl, dbl, D, D, D, D, D, D]),
            "orc_loss_grad": (dbl, [c_int, c_int, c_int, D, D, D, c_int, u64, i64, dbl, dbl, dbl, D, D, D, D]),
            "orc_adam": (None, [i64, D, D, D, D, i64, dbl, dbl, dbl, dbl]),
            "orc_encode": (None, [c_int, c_int, c_int, D, D, D, D, D, D, D, ctypes.POINTER(i64), c_int, u64,
                                  dbl, dbl, dbl, dbl, dbl, D, D, D]),
            "orc_encode_schedule": (None, [c_int, c_int, c_int, D, D, D, D, D, D, D, ctypes.POINTER(i64), c_int,
                                           u64, dbl, dbl, dbl, dbl, dbl, dbl, dbl, i64, dbl, dbl, dbl, D,
                                           D, D]),
            "orc_cdf_q16": (i64, [ctypes.c_int32, i64]),
            "orc_table_entry": (i64, [c_int, c_int]),
            "orc_decode_probs": (None, [c_int, c_int, c_int, I32, F32, I32, I32, U32]),
            "orc_decode_image": (None, [c_int, c_int, c_int, I32, F32, D]),
            "orc_soap_blocks": (c_int, [ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
            "orc_soap_state_count": (i64, []),
            "orc_sym_eig": (None, [c_int, D, D, D]),
            "orc_soap_params": (None, [c_int, D, D, D, D, D, i64, dbl, dbl, dbl, dbl, dbl, dbl, c_int, dbl]),
            "orc_encode_soap": (None, [c_int, c_int, c_int, D, D, D, D, D, D, D, D, ctypes.POINTER(i64), c_int, u64,
                                       dbl, dbl, dbl, dbl, dbl, dbl, dbl, c_int, dbl, D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        assert lib.orc_param_count(0) == N_PARAMS and lib.orc_param_count(1) == N_PARAMS_H
        _lib = lib
        return lib


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------------------------
def _hyper(params) -> int:
    """1 when the parameter vector carries the hyperlatent IFCE block (Sec. III-A3)."""
    n = np.asarray(params).shape[0]
    assert n in (N_PARAMS, N_PARAMS_H), n
    return 1 if n == N_PARAMS_H else 0


def latent_count(H: int, W: int, hyper: bool = False) -> int:
    return int(_load().orc_latent_count(H, W, 1 if hyper else 0))


def grid_shapes(H: int, W: int, hyper: bool = False):
    """Shapes of the latent grids, then (hyper) of the hyperlatent grids (1/16, 1/32, 1/64)."""
    lib = _load()
    out = []
    for k in range(N_GRIDS + (N_HYPER_GRIDS if hyper else 0)):
        h, w = ctypes.c_int(), ctypes.c_int()
        lib.orc_grid_shape(H, W, k, ctypes.byref(h), ctypes.byref(w))
        out.append((h.value, w.value))
    return out


def context_offsets():
    dy = (ctypes.c_int * 16)()
    dx = (ctypes.c_int * 16)()
    _load().orc_context_offsets(dy, dx)
    return list(zip(list(dy), list(dx)))


# ---------------------------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------------------------
def splitmix64_mix(z: int) -> int:
    return int(_load().orc_splitmix64_mix(z))


def noise(seed: int, t: int, n: int) -> np.ndarray:
    lib = _load()
    return np.array([lib.orc_noise(seed, t, i) for i in range(n)], dtype=np.float64)


def gauss(seed: int, t: int, n: int) -> np.ndarray:
    """Box-Muller standard normals of latents 0..n-1 at step t (the soft-round proxy's noise)."""
    lib = _load()
    return np.array([lib.orc_gauss(seed, t, i) for i in range(n)], dtype=np.float64)


def softround(x: float, T: float):
    """(s_T(x), s_T'(x)), Eq. 14."""
    d = ctypes.c_double()
    v = _load().orc_softround(float(x), float(T), ctypes.byref(d))
    return v, d.value


def laplace_prob(y: float, mu: float, b: float):
    dy, dlb = ctypes.c_double(), ctypes.c_double()
    p = _load().orc_laplace_prob(y, mu, b, ctypes.byref(dy), ctypes.byref(dlb))
    return p, dy.value, dlb.value


def upsample(x: np.ndarray, taps, out_shape) -> np.ndarray:
    x = _f64(x)
    taps = _f64(taps)
    th, tw = out_shape
    out = np.zeros((th, tw), dtype=np.float64)
    _load().orc_upsample(x.shape[0], x.shape[1], th, tw, _d(taps), _d(x), _d(out))
    return out


def conv3x3_res(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    x = _f64(x)
    w = _f64(w)
    b = _f64(b)
    out = np.zeros_like(x)
    _load().orc_conv3x3_res(x.shape[1], x.shape[2], _d(w), _d(b), _d(x), _d(out))
    return out


# ---------------------------------------------------------------------------------------------
# whole step
# ---------------------------------------------------------------------------------------------
def forward(image, latents, params, *, lam, mode=MODE_NOISE, seed=0, step=0, sigma=0.0, temp=1.0,
            per_latent=False):
    """Returns dict(loss, rate_bits, mse[, mu, logb, bits, xhat]); sigma and temp are used by
    MODE_SOFTROUND (Eq. 13)."""
    image, latents, params = _f64(image), _f64(latents), _f64(params)
    _, H, W = image.shape
    N = latent_count(H, W, _hyper(params))
    assert latents.shape[0] == N, (latents.shape, N)
    rate, mse = ctypes.c_double(), ctypes.c_double()
    mu = logb = bits = xhat = None
    if per_latent:
        mu, logb, bits = (np.zeros(N) for _ in range(3))
        xhat = np.zeros_like(image)
    loss = _load().orc_forward(H, W, _hyper(params), _d(image), _d(latents), _d(params), mode, seed, step, sigma,
                               temp, lam,
                               ctypes.byref(rate), ctypes.byref(mse), _d(mu), _d(logb), _d(bits),
                               _d(xhat))
    out = dict(loss=loss, rate_bits=rate.value, mse=mse.value)
    if per_latent:
        out.update(mu=mu, logb=logb, bits=bits, xhat=xhat)
    return out


def loss_grad(image, latents, params, *, lam, mode=MODE_NOISE, seed=0, step=0, sigma=0.0, temp=1.0):
    """Returns dict(loss, rate_bits, mse, grad_latents, grad_params)."""
    image, latents, params = _f64(image), _f64(latents), _f64(params)
    _, H, W = image.shape
    assert latents.shape[0] == latent_count(H, W, _hyper(params)), latents.shape
    gy = np.zeros(latents.shape[0])
    gp = np.zeros(params.shape[0])
    rate, mse = ctypes.c_double(), ctypes.c_double()
    loss = _load().orc_loss_grad(H, W, _hyper(params), _d(image), _d(latents), _d(params), mode, seed, step, sigma,
                                 temp,
                                 lam, ctypes.byref(rate), ctypes.byref(mse), _d(gy), _d(gp))
    return dict(loss=loss, rate_bits=rate.value, mse=mse.value, grad_latents=gy, grad_params=gp)


def adam(p, g, m, v, t_new, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam on float64 arrays."""
    _load().orc_adam(p.shape[0], _d(p), _d(_f64(g)), _d(m), _d(v), t_new, lr, b1, b2, eps)


class State:
    """Encoder state held in float64: latents, parameters, Adam moments, step counter."""

    def __init__(self, latents, params, step=0):
        self.latents = _f64(latents).copy()
        self.params = _f64(params).copy()
        self.m_lat = np.zeros_like(self.latents)
        self.v_lat = np.zeros_like(self.latents)
        self.m_par = np.zeros_like(self.params)
        self.v_par = np.zeros_like(self.params)
        self.step = int(step)


def encode(image, state: State, n_iters, *, lam, seed, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
    """Runs n_iters encoder iterations in place on ``state``; returns per-iteration loss/rate/mse."""
    image = _f64(image)
    _, H, W = image.shape
    loss, rate, mse = (np.zeros(n_iters) for _ in range(3))
    step = ctypes.c_int64(state.step)
    _load().orc_encode(H, W, _hyper(state.params), _d(image), _d(state.latents), _d(state.params), _d(state.m_lat),
                       _d(state.v_lat), _d(state.m_par), _d(state.v_par), ctypes.byref(step), n_iters,
                       seed, lam, lr, b1, b2, eps, _d(loss), _d(rate), _d(mse))
    state.step = step.value
    return dict(loss=loss, rate_bits=rate, mse=mse)


def encode_schedule(image, state: State, n_iters, *, lam, seed, n_main, lr_max=1e-2, lr_min=1e-5,
                    sigma0=0.22, sigma1=0.15, temp0=0.35, temp1=0.08, b1=0.9, b2=0.999, eps=1e-8):
    """The paper's encoder schedule (Sec. IV-C/D, Table I) for n_iters iterations from state.step:
    soft-round + Gaussian proxy with linear sigma / T and cosine learning rate over the main stage
    (steps < n_main), then the hard-round stage (latents frozen, parameters at lr_min)."""
    image = _f64(image)
    _, H, W = image.shape
    loss, rate, mse = (np.zeros(n_iters) for _ in range(3))
    step = ctypes.c_int64(state.step)
    _load().orc_encode_schedule(H, W, _hyper(state.params), _d(image), _d(state.latents), _d(state.params),
                                _d(state.m_lat),
                                _d(state.v_lat), _d(state.m_par), _d(state.v_par), ctypes.byref(step), n_iters,
                                seed, lam, lr_max, lr_min, sigma0, sigma1, temp0, temp1, int(n_main), b1, b2, eps,
                                _d(loss), _d(rate), _d(mse))
    state.step = step.value
    return dict(loss=loss, rate_bits=rate, mse=mse)


# ---------------------------------------------------------------------------------------------
# integer decode
# ---------------------------------------------------------------------------------------------
def cdf_q16(s: int, t: int) -> int:
    return int(_load().orc_cdf_q16(int(s), int(t)))


def table_entry(which: int, idx: int) -> int:
    return int(_load().orc_table_entry(which, idx))


def decode_probs(H, W, q_latents, params_f32):
    q = np.ascontiguousarray(q_latents, dtype=np.int32)
    p = np.ascontiguousarray(params_f32, dtype=np.float32)
    N = q.shape[0]
    assert N == latent_count(H, W, _hyper(p)), (N, H, W)
    mu = np.zeros(N, np.int32)
    lb = np.zeros(N, np.int32)
    pr = np.zeros(N, np.uint32)
    _load().orc_decode_probs(H, W, _hyper(p), q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                             mu.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             lb.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             pr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return dict(mu_q=mu, logb_q=lb, prob_q16=pr)


def decode_image(H, W, q_latents, params_f32):
    q = np.ascontiguousarray(q_latents, dtype=np.int32)
    p = np.ascontiguousarray(params_f32, dtype=np.float32)
    assert q.shape[0] == latent_count(H, W, _hyper(p)), (q.shape, H, W)
    out = np.zeros((3, H, W))
    _load().orc_decode_image(H, W, _hyper(p), q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _d(out))
    return out


# ---------------------------------------------------------------------------------------------
# SOAP for the network parameters (Sec. IV-B)
# ---------------------------------------------------------------------------------------------
SOAP_DEFAULTS = dict(b1s=0.95, b2s=0.95, bshamp=0.95, freq=10)


def soap_blocks():
    """[(parameter offset, m, n)] of the two-dimensional blocks that SOAP preconditions."""
    off, m, n = ((ctypes.c_int * 16)() for _ in range(3))
    nb = _load().orc_soap_blocks(off, m, n)
    return [(off[b], m[b], n[b]) for b in range(nb)]


def soap_state_count() -> int:
    return int(_load().orc_soap_state_count())


def sym_eig(A):
    """(Q, lam): eigenvectors as columns of Q, decreasing eigenvalues, canonical signs."""
    A = _f64(A)
    n = A.shape[0]
    Q = np.zeros((n, n))
    lam = np.zeros(n)
    _load().orc_sym_eig(n, _d(np.ascontiguousarray(A)), _d(Q), _d(lam))
    return Q, lam


def soap_params(P, g, m, v, S, t_new, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8, **kw):
    """In-place optimizer step of the parameter vector: SOAP on the 2-D blocks, Adam on the rest."""
    o = dict(SOAP_DEFAULTS, **kw)
    _load().orc_soap_params(_hyper(P), _d(P), _d(_f64(g)), _d(m), _d(v), _d(S), int(t_new), lr, b1, b2, o["b1s"],
                            o["b2s"],
                            o["bshamp"], int(o["freq"]), eps)


def encode_soap(image, state: State, soap_state, n_iters, *, lam, seed, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8, **kw):
    """orc_encode with SOAP on the network parameters; soap_state (float64, soap_state_count())
    is updated in place.  Returns the per-iteration losses."""
    o = dict(SOAP_DEFAULTS, **kw)
    image = _f64(image)
    _, H, W = image.shape
    loss = np.zeros(n_iters)
    step = ctypes.c_int64(state.step)
    _load().orc_encode_soap(H, W, _hyper(state.params), _d(image), _d(state.latents), _d(state.params), _d(state.m_lat), _d(state.v_lat),
                            _d(state.m_par), _d(state.v_par), _d(soap_state), ctypes.byref(step), n_iters, seed, lam,
                            lr, b1, b2, o["b1s"], o["b2s"], o["bshamp"], int(o["freq"]), eps, _d(loss))
    state.step = step.value
    return loss
