"""CPU checks of the C ABI: the library loads, exports every function include/coolchic.h declares,
and its host-side sizing agrees with the oracle and the input generator (no GPU call is made)."""
import ctypes
import os
import re

import pytest

import oracle
from paper_2605_02726_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "coolchic.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(coolchic_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_02726_gb300 import lib as cc
    return cc


def test_library_exports_every_declared_function(lib):
    names = _declared()
    assert len(names) >= 16
    raw = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing
    assert sorted(lib.EXPORTED) == names


def test_host_sizing_agrees_with_oracle_and_generator(lib):
    for H, W in [(64, 64), (512, 768), (1, 1), (37, 53), (2048, 1365)]:
        assert lib.latent_count(H, W) == oracle.latent_count(H, W) == inputs.latent_count(H, W)
        assert [tuple(s) for s in oracle.grid_shapes(H, W)] == inputs.grid_shapes(H, W)
    a = lib.arch(512, 768)
    assert lib.raw().coolchic_param_count(ctypes.byref(a)) == oracle.N_PARAMS == inputs.N_PARAMS
    blocks = lib.param_blocks()
    assert [(n, o, l) for n, o, l in blocks] == [
        (n, inputs.PARAM_OFFSETS[n][0], int(__import__("numpy").prod(s))) for n, s in inputs.PARAM_BLOCKS] + [
        (inputs.HYPER_BLOCK[0], inputs.N_PARAMS, 36)]
    # with hyperlatent grids: three more grids (shapes of grids 4..6) and 36 more parameters
    ah = lib.arch(512, 768, hyper=True)
    assert lib.raw().coolchic_param_count(ctypes.byref(ah)) == oracle.N_PARAMS_H == inputs.N_PARAMS_H
    for H, W in [(64, 64), (37, 53), (1, 1), (2048, 1365)]:
        assert lib.latent_count(H, W, True) == oracle.latent_count(H, W, True) == inputs.latent_count(H, W, True)
        assert [tuple(s) for s in oracle.grid_shapes(H, W, True)] == inputs.grid_shapes(H, W, hyper=True)
    ah.hyper_grids = 2
    assert lib.raw().coolchic_latent_count(ctypes.byref(ah)) == -1


def test_argument_checks_fail_cleanly(lib):
    raw = lib.raw()
    a = lib.Arch()
    assert raw.coolchic_arch_init(ctypes.byref(a), 0, 10) == -1
    assert b"outside" in raw.coolchic_last_error()
    assert raw.coolchic_arch_init(ctypes.byref(a), 64, 64) == 0
    a.L = 5
    assert raw.coolchic_latent_count(ctypes.byref(a)) == -1
    assert b"architecture" in raw.coolchic_last_error()
    assert raw.coolchic_param_block(99, None, None, None) == -1
    assert raw.coolchic_version().startswith(b"coolchic")


def test_launch_count_and_init_state_argument_checks(lib):
    raw = lib.raw()
    a = lib.arch(512, 768)
    # relax once per call, then 13 kernels per iteration
    assert [raw.coolchic_kernel_launches(ctypes.byref(a), n) for n in (0, 1, 3)] == [0, 14, 40]
    assert raw.coolchic_kernel_launches(ctypes.byref(a), -1) == -1
    # NULL state pointers and a bad architecture are refused before any device call
    st = lib.State()
    assert raw.coolchic_init_state(ctypes.byref(a), 1, ctypes.byref(st), None) == -1
    assert b"NULL" in raw.coolchic_last_error()
    assert raw.coolchic_init_state(None, 1, ctypes.byref(st), None) == -1
