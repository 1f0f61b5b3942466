"""The sampled-row oracle equals the full tier-2 sigma on the rows it computes."""
import numpy as np
import pytest

from adc_inputs import make_system
from oracle.sampled import sigma_ea_rows
from oracle.spinadapted import SpinAdaptedADC


@pytest.mark.parametrize("order", [2, 3])
def test_sampled_rows_match_full_sigma(order):
    o, v, naux = 5, 17, 30
    s = make_system(o, v, naux, seed=2)
    T = SpinAdaptedADC(s.eps, o, s.B, order, "ea")
    x = np.random.default_rng(3).standard_normal(T.dim)
    full = T.sigma(x)[v:].reshape(o, v, v)
    rows = [0, 2, 4]
    got = sigma_ea_rows(s.eps, s.B, o, x[:v], x[v:].reshape(o, v, v), rows, order=order)
    assert np.abs(got - full[rows]).max() < 1e-12 * np.abs(full).max()


@pytest.mark.parametrize("order", [2, 3])
def test_sampled_rows_without_1p_part(order):
    """With y1 = 0 the terms linear in y1 are skipped (no full amplitudes formed); the rows
    still equal the full sigma of that vector."""
    o, v, naux = 4, 15, 28
    s = make_system(o, v, naux, seed=5)
    T = SpinAdaptedADC(s.eps, o, s.B, order, "ea")
    x = np.random.default_rng(4).standard_normal(T.dim)
    x[:v] = 0.0
    full = T.sigma(x)[v:].reshape(o, v, v)
    rows = [1, 3]
    got = sigma_ea_rows(s.eps, s.B, o, x[:v], x[v:].reshape(o, v, v), rows, order=order)
    assert np.abs(got - full[rows]).max() < 1e-12 * np.abs(full).max()
