"""heat_debye_enthalpy through the C ABI (host function, no GPU needed).

The bins of the method sit on a temperature grid with enthalpies E_i = H(T_i) (Sec. 2);
the library's helper gives the Debye H(T).  Pinned against the model's two closed-form
limits (with their next correction terms), an independent adaptive quadrature of the
Debye integral, and the input generator's own H(T)."""
import math
import shutil

import numpy as np
import pytest

from paper_1311_4627_gb300 import build, heat
from paper_1311_4627_gb300 import workloads as W

K = 1.380649e-16


@pytest.fixture(scope="module")
def L():
    if shutil.which("nvcc") is None and not __import__("os").path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    build.build_lib()
    return heat.lib()


@pytest.mark.parametrize("theta", [420.0, 500.0])
def test_low_temperature_limit(L, theta):
    """T << theta: H = (3 pi^4 / 5) N k T^4 / theta^3 (the T^3 heat capacity integrated);
    the neglected tail is below y^3 e^-y of the integral, y = theta/T >= 50."""
    n = 1234.5
    for y in (50.0, 80.0, 200.0, 1e4):
        T = theta / y
        ref = 3.0 * math.pi**4 / 5.0 * n * K * T**4 / theta**3
        got = L.heat_debye_enthalpy(theta, n, T)
        assert abs(got / ref - 1.0) < 1e-13, (y, got, ref)


@pytest.mark.parametrize("theta", [420.0, 500.0])
def test_high_temperature_limit(L, theta):
    """T >> theta: H = 3 N k T - (9/8) N k theta + (3/20) N k theta^2 / T + O(y^4 N k T):
    a wrong prefactor, power of T or sign of the zero-point-free offset fails this."""
    n = 7.0e5
    for y in (1e-3, 1e-2, 5e-2, 0.2):
        T = theta / y
        ref = 3.0 * n * K * T - 9.0 / 8.0 * n * K * theta + 3.0 / 20.0 * n * K * theta**2 / T
        got = L.heat_debye_enthalpy(theta, n, T)
        assert abs(got / ref - 1.0) <= y**4 / 1500.0 + 1e-14, (y, got / ref - 1.0)


def test_against_adaptive_quadrature(L):
    """The Debye integral by scipy's adaptive quadrature at theta/T from 1e-3 to 300,
    including both sides of the switch between the two series at theta/T = 1."""
    integrate = pytest.importorskip("scipy.integrate")
    theta, n = 420.0, 3.3e3
    ys = np.concatenate([np.geomspace(1e-3, 300.0, 37), [1.0 - 1e-9, 1.0, 1.0 + 1e-9]])
    for y in ys:
        f = lambda x: x**3 / math.expm1(x) if x > 0 else 0.0  # noqa: E731
        D, _ = integrate.quad(f, 0.0, y, epsabs=0.0, epsrel=2e-14, limit=200)
        T = theta / y
        ref = 9.0 * n * K * T * (T / theta) ** 3 * D
        got = L.heat_debye_enthalpy(theta, n, T)
        assert abs(got / ref - 1.0) < 2e-13, (y, got / ref - 1.0)


def test_matches_the_input_generator(L):
    """The workloads' bins (config grids) can be built through the library: same H(T)."""
    for comp in ("carbonaceous", "silicate"):
        theta = W.COMPOSITIONS[comp][0]
        for a_um in (3.5e-4, 0.01, 1.0):
            n = W.n_atoms(a_um * W.UM, comp)
            T = np.geomspace(2.7, 2500.0, 64)
            ref = W.debye_enthalpy(theta, n, T)
            got = heat.heat_debye_enthalpy(theta, n, T)
            np.testing.assert_allclose(got, ref, rtol=1e-11, atol=0.0)
            assert np.all(np.diff(got) > 0.0)


def test_bad_arguments_give_nan_and_zero_at_zero_temperature(L):
    assert L.heat_debye_enthalpy(420.0, 10.0, 0.0) == 0.0
    for args in ((0.0, 10.0, 5.0), (-1.0, 10.0, 5.0), (420.0, 0.0, 5.0), (420.0, 10.0, -1.0),
                 (float("nan"), 10.0, 5.0), (420.0, float("inf"), 5.0), (420.0, 10.0, float("inf"))):
        assert math.isnan(L.heat_debye_enthalpy(*args)), args
