"""Spectral function of computed roots (Sec. II A, Eqs. g_adc and spec_function;
Sec. IV, Eq. PES).  TEST INFRASTRUCTURE ONLY -- nothing in the GPU product path
may import this module.

* ``propagator``: G(w) = X (w 1 - Omega + i eta)^-1 X^dagger for spectroscopic
  amplitudes X [nmo, nroots] and root energies Omega (Eq. g_adc, evaluated at
  w + i eta).
* ``spectral_function``: A(w) = -1/pi Im Tr G(w) (Eq. spec_function), from the
  explicit propagator.
* ``dos``: A(w) = -1/pi Im sum_mu P_mu / (w - w_mu + i eta) from spectroscopic
  factors (Eq. PES).
"""
from __future__ import annotations

import numpy as np


def propagator(X, energies, w, eta):
    """G_pq(w) for X [nmo, nroots] (complex, [nmo, nmo])."""
    X = np.asarray(X, dtype=np.float64)
    d = 1.0 / (w - np.asarray(energies, dtype=np.float64) + 1j * eta)
    return (X * d[None, :]) @ X.T


def spectral_function(X, energies, omega, eta):
    return np.array([-np.trace(propagator(X, energies, w, eta)).imag / np.pi for w in np.atleast_1d(omega)])


def dos(energies, P, omega, eta):
    omega = np.atleast_1d(np.asarray(omega, dtype=np.float64))
    z = omega[:, None] - np.asarray(energies, dtype=np.float64)[None, :] + 1j * eta
    return -(np.asarray(P, dtype=np.float64)[None, :] / z).sum(axis=1).imag / np.pi
