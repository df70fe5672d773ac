"""Thin ctypes binding of libcoolchic.so (include/coolchic.h).

Argument marshalling only: torch tensors supply device memory and streams, every computation
runs in the library's CUDA kernels.  There is no CPU fallback; if the library cannot be loaded
the import fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcoolchic.so")

CC_OK = 0
CC_RELAX_NOISE, CC_RELAX_HARD, CC_RELAX_IDENTITY = 0, 1, 2
N_GRIDS = 7
N_PARAMS = 1415


class Arch(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("C", "H", "W", "L", "n_ctx", "ifce_dim", "ifce_grids",
                                              "arm_hidden", "arm_layers", "syn_hidden", "n_resconv",
                                              "up_taps", "stabilizer", "hyper_grids")]


class HParams(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_float), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("noise_mode", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("sigma0", ctypes.c_float), ("sigma1", ctypes.c_float),
                ("temp0", ctypes.c_float), ("temp1", ctypes.c_float), ("lr_min", ctypes.c_float),
                ("nn_optimizer", ctypes.c_int32), ("n_main", ctypes.c_int64), ("soap_beta1", ctypes.c_float),
                ("soap_beta2", ctypes.c_float), ("soap_shampoo_beta", ctypes.c_float), ("soap_freq", ctypes.c_int32)]


class State(ctypes.Structure):
    _fields_ = [("latents", ctypes.c_void_p), ("params", ctypes.c_void_p), ("m_lat", ctypes.c_void_p),
                ("v_lat", ctypes.c_void_p), ("m_par", ctypes.c_void_p), ("v_par", ctypes.c_void_p),
                ("step", ctypes.c_void_p), ("soap", ctypes.c_void_p)]


class RD(ctypes.Structure):
    _fields_ = [("loss", ctypes.c_double), ("rate_bits", ctypes.c_double), ("mse", ctypes.c_double)]


class Schedule(ctypes.Structure):
    """Per kernel class, the fraction (0, 1] of each job's single-image CTA count used in a batch."""
    _fields_ = [("arm", ctypes.c_float), ("syn", ctypes.c_float), ("conv", ctypes.c_float), ("other", ctypes.c_float)]

    def as_tuple(self):
        return (self.arm, self.syn, self.conv, self.other)


class CoolChicError(RuntimeError):
    pass


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2605_02726_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp, i32, i64, sz, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_float
    sig = {
        "coolchic_arch_init": (i32, [P(Arch), i32, i32]),
        "coolchic_latent_count": (i64, [P(Arch)]),
        "coolchic_param_count": (i64, [P(Arch)]),
        "coolchic_init_state": (i32, [P(Arch), ctypes.c_uint64, P(State), vp]),
        "coolchic_param_block": (i32, [i32, P(ctypes.c_char_p), P(i32), P(i32)]),
        "coolchic_workspace_bytes": (sz, [P(Arch), i32]),
        "coolchic_kernel_launches": (i64, [P(Arch), i32]),
        "coolchic_encode_step": (i32, [P(Arch), P(HParams), vp, P(State), i32, vp, vp, sz, vp]),
        "coolchic_encode_step_host": (i32, [P(Arch), P(HParams), vp, P(State), i32, vp, vp, sz, vp]),
        "coolchic_forward": (i32, [P(Arch), P(HParams), vp, vp, vp, i64, i32, i32, vp, vp, vp, sz, vp]),
        "coolchic_backward": (i32, [P(Arch), P(HParams), vp, vp, vp, i64, i32, i32, f32, vp, vp, vp, sz, vp]),
        "coolchic_rate_distortion": (i32, [P(Arch), P(HParams), vp, vp, vp, i64, i32, P(RD), vp, sz, vp]),
        "coolchic_decode_image": (i32, [P(Arch), vp, vp, vp, vp, vp, vp, vp, sz, vp]),
        "coolchic_rate_distortion_noalloc": (i32, [P(Arch), P(HParams), vp, vp, vp, i64, i32, P(RD), vp]),
        "coolchic_batch_table_bytes": (sz, [i32, i32]),
        "coolchic_batch_create": (i32, [i32, vp, vp, vp, vp, vp, vp, P(Schedule), i32, vp, sz, P(vp)]),
        "coolchic_batch_create_async": (i32, [i32, vp, vp, vp, vp, vp, vp, P(Schedule), i32, vp, sz, vp, vp, P(vp)]),
        "coolchic_batch_step": (i32, [vp, i32, vp]),
        "coolchic_batch_records": (vp, [vp]),
        "coolchic_batch_destroy": (i32, [vp]),
        "coolchic_timing_enable": (i32, [i32, i32]),
        "coolchic_timing_collect": (i32, [P(ctypes.c_double), P(i64)]),
        "coolchic_timing_disable": (i32, []),
        "coolchic_measure_peak": (i32, [i32, vp, P(ctypes.c_double), P(ctypes.c_double), vp]),
        "coolchic_soap_state_floats": (i64, []),
        "coolchic_test_inject_stall": (i32, [i32]),
        "coolchic_last_error": (ctypes.c_char_p, []),
        "coolchic_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ["coolchic_arch_init", "coolchic_latent_count", "coolchic_param_count", "coolchic_init_state",
            "coolchic_param_block",
            "coolchic_workspace_bytes", "coolchic_kernel_launches", "coolchic_encode_step", "coolchic_forward", "coolchic_backward",
            "coolchic_rate_distortion", "coolchic_decode_image", "coolchic_timing_enable", "coolchic_timing_collect",
            "coolchic_timing_disable", "coolchic_last_error", "coolchic_version",
            "coolchic_rate_distortion_noalloc", "coolchic_batch_table_bytes", "coolchic_batch_create",
            "coolchic_batch_step", "coolchic_batch_records", "coolchic_batch_destroy", "coolchic_measure_peak",
            "coolchic_encode_step_host", "coolchic_soap_state_floats",
            "coolchic_batch_create_async", "coolchic_test_inject_stall"]

KERNEL_ARM, KERNEL_SYN_BWD, KERNEL_CONV, KERNEL_SYN_FWD = 0, 1, 2, 3
KERNEL_UP_FWD, KERNEL_UP_ADJ, KERNEL_GATHER = 4, 5, 6


def timing_enable(kernel_id: int, max_launches: int):
    _check(_lib.coolchic_timing_enable(kernel_id, max_launches), "timing_enable")


def timing_collect():
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(_lib.coolchic_timing_collect(ctypes.byref(ms), ctypes.byref(n)), "timing_collect")
    return ms.value, n.value


def timing_disable():
    _lib.coolchic_timing_disable()


PEAK_FP32_FMA, PEAK_TF32_MMA = 0, 1


def measure_peak(which: int, stream=None):
    """Measured throughput ceiling of one pipe on the current device: (TFLOP/s, ms of the timed
    launch).  Blocking."""
    import torch
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.coolchic_measure_peak(int(which), _ptr(sink), ctypes.byref(tf), ctypes.byref(ms), _stream(stream)),
           "measure_peak")
    return tf.value, ms.value


def raw():
    """The ctypes library handle (for tests of the C ABI itself)."""
    return _lib


def _check(rc: int, what: str):
    if rc != CC_OK:
        raise CoolChicError(f"{what} failed ({rc}): {_lib.coolchic_last_error().decode()}")


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t):
    if t is None:
        return None
    if t.device.type != "cpu" or not t.is_contiguous():
        raise ValueError("expected a contiguous host tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


N_PARAMS_H = 1451  # with hyperlatent grids: + the IFCE weights of their inputs
N_HYPER_GRIDS = 3


def arch(H: int, W: int, hyper: bool = False) -> Arch:
    """The library's architecture for an H x W image; hyper: three hyperlatent grids (Sec. III-A3)."""
    a = Arch()
    _check(_lib.coolchic_arch_init(ctypes.byref(a), H, W), "arch_init")
    a.hyper_grids = N_HYPER_GRIDS if hyper else 0
    return a


def _hy(params) -> bool:
    """A parameter vector of 1451 values carries the hyperlatent IFCE block."""
    return int(params.numel()) == N_PARAMS_H


CC_NOISE_UNIFORM, CC_NOISE_SOFTROUND = 0, 1


CC_OPT_ADAM, CC_OPT_SOAP = 0, 1
# SOAP settings (the SOAP paper's defaults; the Cool-chic paper gives none): moment betas,
# preconditioner beta, eigenbasis refresh period
SOAP_DEFAULTS = dict(soap_beta1=0.95, soap_beta2=0.95, soap_shampoo_beta=0.95, soap_freq=10)


def _with_soap(hp: HParams, soap: bool, **kw) -> HParams:
    o = dict(SOAP_DEFAULTS, **kw)
    hp.nn_optimizer = CC_OPT_SOAP if soap else CC_OPT_ADAM
    hp.soap_beta1, hp.soap_beta2 = o["soap_beta1"], o["soap_beta2"]
    hp.soap_shampoo_beta, hp.soap_freq = o["soap_shampoo_beta"], int(o["soap_freq"])
    return hp


def hparams(lam=1e-3, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, seed=0, soap=False, **soap_kw) -> HParams:
    """Additive uniform proxy, constant learning rate; soap=True: SOAP on the network's 2-D blocks."""
    return _with_soap(HParams(lam, lr, beta1, beta2, eps, CC_NOISE_UNIFORM, seed, 0.0, 0.0, 1.0, 1.0, lr, 0, 0),
                      soap, **soap_kw)


def hparams_schedule(lam=1e-3, n_main=1000, lr=1e-2, lr_min=1e-5, sigma0=0.22, sigma1=0.15, temp0=0.35,
                     temp1=0.08, beta1=0.9, beta2=0.999, eps=1e-8, seed=0, soap=False, **soap_kw) -> HParams:
    """The paper's soft-round proxy and schedule (Table I defaults): main stage for steps < n_main,
    then the hard-round stage."""
    return _with_soap(HParams(lam, lr, beta1, beta2, eps, CC_NOISE_SOFTROUND, seed, sigma0, sigma1, temp0, temp1,
                              lr_min, 0, int(n_main)), soap, **soap_kw)


def soap_state_floats() -> int:
    return int(_lib.coolchic_soap_state_floats())


def latent_count(H: int, W: int, hyper: bool = False) -> int:
    return int(_lib.coolchic_latent_count(ctypes.byref(arch(H, W, hyper))))


def kernel_launches(H: int, W: int, n_iters: int) -> int:
    """Kernel launches of one encode_step call of n_iters iterations on an H x W image."""
    return int(_lib.coolchic_kernel_launches(ctypes.byref(arch(H, W)), int(n_iters)))


def param_blocks():
    out = []
    i = 0
    while True:
        name = ctypes.c_char_p()
        off, ln = ctypes.c_int32(), ctypes.c_int32()
        if _lib.coolchic_param_block(i, ctypes.byref(name), ctypes.byref(off), ctypes.byref(ln)) != CC_OK:
            break
        out.append((name.value.decode(), off.value, ln.value))
        i += 1
    return out


def workspace(H: int, W: int, store_activations: bool = False, device=None, host_io: bool = False,
              hyper: bool = False) -> torch.Tensor:
    """Device workspace for one job (256-byte aligned byte tensor); host_io adds the room
    encode_step_host needs."""
    flags = (1 if store_activations else 0) | (2 if host_io else 0)
    n = int(_lib.coolchic_workspace_bytes(ctypes.byref(arch(H, W, hyper)), flags))
    if n == 0:
        raise CoolChicError(_lib.coolchic_last_error().decode())
    buf = torch.empty(n + 256, dtype=torch.uint8, device=device or "cuda")
    off = (-buf.data_ptr()) % 256
    return buf[off:off + n]


class EncoderState:
    """Device-resident encoder state: latents, parameters, Adam moments, step counter."""

    def __init__(self, latents: torch.Tensor, params: torch.Tensor, step: int = 0, soap: bool = False):
        dev = latents.device
        self.latents = latents.detach().clone().float().contiguous()
        self.params = params.detach().clone().float().contiguous()
        self.m_lat = torch.zeros_like(self.latents)
        self.v_lat = torch.zeros_like(self.latents)
        self.m_par = torch.zeros_like(self.params)
        self.v_par = torch.zeros_like(self.params)
        self.step = torch.full((1,), int(step), dtype=torch.int64, device=dev)
        # SOAP preconditioners and eigenbases (L, R, Q_L, Q_R of every 2-D block), zero at the start
        self.soap = torch.zeros(soap_state_floats(), device=dev) if soap else None

    def c_state(self) -> State:
        return State(self.latents.data_ptr(), self.params.data_ptr(), self.m_lat.data_ptr(), self.v_lat.data_ptr(),
                     self.m_par.data_ptr(), self.v_par.data_ptr(), self.step.data_ptr(),
                     self.soap.data_ptr() if self.soap is not None else None)

    @staticmethod
    def init(H: int, W: int, seed: int, device=None, stream=None, hyper: bool = False, soap: bool = False) -> "EncoderState":
        """A fresh state initialised on the device by coolchic_init_state (seeded: latents
        0.01 N(0, 1), hidden weights U(+-1/sqrt(fan_in)), bicubic taps, the rest zero)."""
        dev = torch.device(device or "cuda")
        a = arch(H, W, hyper)
        n_par = int(_lib.coolchic_param_count(ctypes.byref(a)))
        st = EncoderState(torch.empty(latent_count(H, W, hyper), device=dev), torch.empty(n_par, device=dev),
                          soap=soap)
        cs = st.c_state()
        _check(_lib.coolchic_init_state(ctypes.byref(a), int(seed), ctypes.byref(cs), _stream(stream)), "init_state")
        return st

    def clone(self) -> "EncoderState":
        s = EncoderState.__new__(EncoderState)
        for k in ("latents", "params", "m_lat", "v_lat", "m_par", "v_par", "step"):
            setattr(s, k, getattr(self, k).clone())
        s.soap = self.soap.clone() if self.soap is not None else None
        return s


def encode_step(image, state: EncoderState, n_iters: int, *, H, W, hp: HParams, ws, rd=None, stream=None):
    """n_iters encoder iterations in place; rd (optional, float64 [n_iters, 3]) gets loss/rate/mse."""
    a = arch(H, W, _hy(state.params))
    cs = state.c_state()
    _check(_lib.coolchic_encode_step(ctypes.byref(a), ctypes.byref(hp), _ptr(image), ctypes.byref(cs), n_iters,
                                     _ptr(rd), _ptr(ws), ws.numel(), _stream(stream)), "encode_step")


def encode_step_host(image_host, state: EncoderState, n_iters: int, *, H, W, hp: HParams, ws, rd_host=None,
                     stream=None):
    """encode_step on a host image (CPU tensor, pinned for an asynchronous copy); the last
    iteration's (loss, rate, mse) lands in rd_host (CPU float64 [3], nullable) once the stream has
    reached it.  ws must come from workspace(..., host_io=True)."""
    a = arch(H, W, _hy(state.params))
    cs = state.c_state()
    _check(_lib.coolchic_encode_step_host(ctypes.byref(a), ctypes.byref(hp), _host_ptr(image_host), ctypes.byref(cs),
                                          n_iters, _host_ptr(rd_host), _ptr(ws), ws.numel(), _stream(stream)),
           "encode_step_host")


def forward(image, latents, params, *, H, W, hp: HParams, step=0, relax=CC_RELAX_NOISE, ws, store=False,
            rd=None, xhat=None, stream=None):
    a = arch(H, W, _hy(params))
    _check(_lib.coolchic_forward(ctypes.byref(a), ctypes.byref(hp), _ptr(image), _ptr(latents), _ptr(params),
                                 int(step), relax, 1 if store else 0, _ptr(rd), _ptr(xhat), _ptr(ws), ws.numel(),
                                 _stream(stream)), "forward")


def backward(image, latents, params, grad_latents, grad_params, *, H, W, hp: HParams, step=0,
             relax=CC_RELAX_NOISE, ws, use_stored=False, grad_scale=1.0, stream=None):
    a = arch(H, W, _hy(params))
    _check(_lib.coolchic_backward(ctypes.byref(a), ctypes.byref(hp), _ptr(image), _ptr(latents), _ptr(params),
                                  int(step), relax, 1 if use_stored else 0, float(grad_scale), _ptr(grad_latents),
                                  _ptr(grad_params), _ptr(ws), ws.numel(), _stream(stream)), "backward")


def rate_distortion(image, latents, params, *, H, W, hp: HParams, step=0, relax=CC_RELAX_HARD, ws, stream=None):
    a = arch(H, W, _hy(params))
    out = RD()
    _check(_lib.coolchic_rate_distortion(ctypes.byref(a), ctypes.byref(hp), _ptr(image), _ptr(latents),
                                         _ptr(params), int(step), relax, ctypes.byref(out), _ptr(ws), ws.numel(),
                                         _stream(stream)), "rate_distortion")
    return dict(loss=out.loss, rate_bits=out.rate_bits, mse=out.mse)


def rate_distortion_noalloc(image, latents, params, *, H, W, hp: HParams, step=0, relax=CC_RELAX_HARD,
                            stream=None):
    """coolchic_rate_distortion without a workspace: for callers that cannot allocate device
    memory (the library's built-in scratch is used; images up to about 1.4 million pixels)."""
    a = arch(H, W)
    out = RD()
    _check(_lib.coolchic_rate_distortion_noalloc(ctypes.byref(a), ctypes.byref(hp), _ptr(image), _ptr(latents),
                                                 _ptr(params), int(step), relax, ctypes.byref(out),
                                                 _stream(stream)), "rate_distortion_noalloc")
    return dict(loss=out.loss, rate_bits=out.rate_bits, mse=out.mse)


def decode_image(q_latents, params, *, H, W, ws, image_out=None, prob=None, mu_q=None, logb_q=None, stream=None):
    a = arch(H, W, _hy(params))
    _check(_lib.coolchic_decode_image(ctypes.byref(a), _ptr(q_latents), _ptr(params), _ptr(image_out), _ptr(prob),
                                      _ptr(mu_q), _ptr(logb_q), _ptr(ws), ws.numel(), _stream(stream)),
           "decode_image")


class BatchEncoder:
    """Encoder iterations of many images in one set of launches (coolchic_batch_*).

    jobs: list of (image [3,H,W] CUDA float32, EncoderState, HParams).  Each job keeps its own
    workspace; the plan table lives in a device buffer owned by this object.  `step(n)` is
    asynchronous; `graph(n)` captures n iterations in a CUDA graph for replay."""

    def __init__(self, jobs, schedule=None, rd_capacity=1, device=None, workspaces=None, stream=None):
        """stream: plan without blocking (coolchic_batch_create_async): the table is copied on
        that stream from a pinned staging buffer, and the batch's steps must run on it."""
        self.jobs = list(jobs)
        n = len(self.jobs)
        if n == 0:
            raise ValueError("empty batch")
        self.shapes = [(int(img.shape[1]), int(img.shape[2])) for img, _, _ in self.jobs]
        dev = device or self.jobs[0][0].device
        self.workspaces = list(workspaces) if workspaces is not None else [
            workspace(H, W, device=dev, hyper=_hy(st.params)) for (H, W), (_, st, _) in zip(self.shapes, self.jobs)]
        archs = (Arch * n)(*[arch(H, W, _hy(st.params)) for (H, W), (_, st, _) in zip(self.shapes, self.jobs)])
        hps = (HParams * n)(*[hp for _, _, hp in self.jobs])
        images = (ctypes.c_void_p * n)(*[img.data_ptr() for img, _, _ in self.jobs])
        states = (State * n)(*[st.c_state() for _, st, _ in self.jobs])
        wss = (ctypes.c_void_p * n)(*[w.data_ptr() for w in self.workspaces])
        wsb = (ctypes.c_size_t * n)(*[w.numel() for w in self.workspaces])
        tb = int(_lib.coolchic_batch_table_bytes(n, rd_capacity))
        buf = torch.empty(tb + 256, dtype=torch.uint8, device=dev)
        off = (-buf.data_ptr()) % 256
        self.table = buf[off:off + tb]
        self.rd_capacity = rd_capacity
        self.schedule = schedule
        handle = ctypes.c_void_p()
        sched = ctypes.byref(schedule) if schedule is not None else None
        if stream is None:
            torch.cuda.synchronize(dev)
            _check(_lib.coolchic_batch_create(n, archs, hps, images, states, wss, wsb, sched, rd_capacity,
                                              ctypes.c_void_p(self.table.data_ptr()), tb, ctypes.byref(handle)),
                   "batch_create")
        else:
            self.staging = torch.empty(tb, dtype=torch.uint8).pin_memory()  # kept alive with the batch
            _check(_lib.coolchic_batch_create_async(n, archs, hps, images, states, wss, wsb, sched, rd_capacity,
                                                    ctypes.c_void_p(self.table.data_ptr()), tb,
                                                    ctypes.c_void_p(self.staging.data_ptr()), _stream(stream),
                                                    ctypes.byref(handle)), "batch_create_async")
        self.handle = handle

    def step(self, n_iters=1, stream=None):
        _check(_lib.coolchic_batch_step(self.handle, int(n_iters), _stream(stream)), "batch_step")

    def records(self):
        """float64 [rd_capacity, n_jobs, 3] view (loss, rate_bits, mse) of the last step call."""
        ptr = _lib.coolchic_batch_records(self.handle)
        off = ptr - self.table.data_ptr()
        n = len(self.jobs)
        return self.table[off:off + self.rd_capacity * n * 24].view(torch.float64).view(self.rd_capacity, n, 3)

    def graph(self, n_iters=1):
        s = torch.cuda.Stream(device=self.table.device)
        s.wait_stream(torch.cuda.current_stream(self.table.device))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.step(n_iters, stream=s)
        return g

    def close(self):
        if getattr(self, "handle", None):
            _lib.coolchic_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
