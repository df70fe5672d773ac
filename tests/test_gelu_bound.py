"""The synthesis kernels evaluate GELU's Gaussian CDF through Abramowitz & Stegun formula 7.1.26.

These CPU checks pin the published bound of that approximation (|error| <= 1.5e-7 on erf) and the
two identities the kernels rely on: Phi(-|a|) is taken straight from the erfc product, and the GELU
derivative reuses exp(-a^2/2).  The kernels themselves are checked against the FP64 oracle (exact
erf) by the GPU parity tests.
"""
import numpy as np
import pytest
from scipy.special import erf, erfc

P = 0.3275911
A = (0.254829592, -0.284496736, 1.421413741, -1.453152027, 1.061405429)


def erfc_as(x):
    s = 1.0 / (1.0 + P * x)
    q = s * (A[0] + s * (A[1] + s * (A[2] + s * (A[3] + s * A[4]))))
    return q * np.exp(-x * x)


def gelu_as(a):
    lt = 0.5 * erfc_as(np.abs(a) / np.sqrt(2.0))
    phi = np.where(a < 0, lt, 1.0 - lt)
    return a * phi, phi + a * np.exp(-0.5 * a * a) / np.sqrt(2.0 * np.pi)


def test_erf_error_bound():
    x = np.linspace(0.0, 12.0, 2_000_001)
    err = np.abs((1.0 - erfc_as(x)) - erf(x))
    assert err.max() <= 1.5e-7
    assert err.max() > 1e-8  # the bound is tight enough to mean something


@pytest.mark.parametrize("a", [-8.0, -3.0, -0.5, 0.0, 0.25, 1.0, 4.0, 9.0])
def test_gelu_and_derivative(a):
    g, dg = gelu_as(np.float64(a))
    g_ref = 0.5 * a * (1.0 + erf(a / np.sqrt(2.0)))
    assert abs(g - g_ref) <= 0.5 * abs(a) * 1.5e-7 + 1e-300
    h = 1e-5
    fd = (0.5 * (a + h) * erfc(-(a + h) / np.sqrt(2.0)) - 0.5 * (a - h) * erfc(-(a - h) / np.sqrt(2.0))) / (2 * h)
    assert abs(dg - fd) <= 2e-7


def test_lower_tail_has_no_cancellation():
    # Phi(-5) = 2.87e-7: the product form keeps ~1e-2 relative accuracy where 1 + erf(-x) in FP32
    # would keep none.
    a = -5.0
    lt = 0.5 * erfc_as(abs(a) / np.sqrt(2.0))
    ref = 0.5 * erfc(abs(a) / np.sqrt(2.0))
    assert abs(lt - ref) / ref < 0.05
