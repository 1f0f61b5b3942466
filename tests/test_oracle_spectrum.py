"""Pins of the spectral-function oracle (Eqs. g_adc, spec_function, PES) and the
library's adc_spectrum (host computation, no GPU needed).

* One pole: A(w_mu) = P / (pi eta) (closed form of the Lorentzian peak).
* Integral over [a, b]: sum_mu P_mu (arctan((b - w_mu)/eta) - arctan((a - w_mu)/eta)) / pi,
  the closed-form antiderivative, against a fine trapezoid of the oracle.
* Trace identity: -1/pi Im Tr[X (w - Omega + i eta)^-1 X^T] equals the P form with
  P_mu = sum_p X_{p mu}^2 (Eq. spec_factors).
* adc_spectrum reproduces the oracle to rounding and rejects bad arguments.
"""
import numpy as np
import pytest

from oracle.spectrum import dos, propagator, spectral_function


def test_single_pole_peak():
    assert abs(dos([0.3], [1.7], 0.3, 0.05)[0] - 1.7 / (np.pi * 0.05)) < 1e-12


def test_integral_closed_form():
    rng = np.random.default_rng(1)
    e, P, eta = rng.uniform(-1, 1, 5), rng.uniform(0, 2, 5), 0.02
    a, b = -3.0, 3.0
    w = np.linspace(a, b, 600001)
    A = dos(e, P, w, eta)
    num = np.sum(0.5 * (A[1:] + A[:-1]) * np.diff(w))
    exact = np.sum(P * (np.arctan((b - e) / eta) - np.arctan((a - e) / eta))) / np.pi
    assert abs(num - exact) < 1e-6 * exact


def test_trace_identity():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((7, 4))
    e = rng.uniform(-1, 1, 4)
    w = np.linspace(-2, 2, 41)
    A1 = spectral_function(X, e, w, 0.1)
    A2 = dos(e, (X * X).sum(axis=0), w, 0.1)
    assert np.abs(A1 - A2).max() < 1e-12
    G = propagator(X, e, 0.37, 0.1)
    assert np.abs(G - G.T).max() < 1e-14  # symmetric for real X


def test_library_spectrum_matches_oracle():
    from paper_2012_06714_gb300 import spectrum

    rng = np.random.default_rng(3)
    e, P = rng.uniform(-1, 1, 6), rng.uniform(0, 2, 6)
    w = np.linspace(-1.5, 1.5, 301)
    assert np.abs(spectrum(e, P, w, 0.03) - dos(e, P, w, 0.03)).max() < 1e-12
    assert spectrum([], [], w, 0.03).max() == 0.0


def test_library_spectrum_rejects_bad_arguments():
    from paper_2012_06714_gb300 import spectrum
    from paper_2012_06714_gb300._lib import ADCError

    with pytest.raises(ADCError):
        spectrum([0.1], [1.0], [0.0], 0.0)
    with pytest.raises(ValueError):
        spectrum([0.1, 0.2], [1.0], [0.0], 0.1)
