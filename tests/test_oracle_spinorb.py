"""Tier-1 (explicit spin-orbital equations) against tier 0 (operator definitions),
block by block: every ADC matrix element and transition moment, EA and IP, n = 2, 3."""
import numpy as np
import pytest

from adc_inputs import make_system
from oracle.fock import ADCFock
from oracle.spinorb import SpinOrbitalADC

CASES = [(2, 3, 5), (3, 3, 6), (2, 4, 7)]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"o{c[0]}v{c[1]}")
def pair(request):
    o, v, seed = request.param
    s = make_system(o, v, 12, seed=seed)
    B = 2.0 * s.B
    return ADCFock(s.eps, o, 3, B=B), s, B


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_matrix_adc3(pair, kind):
    F, s, B = pair
    M, _ = F.adc_matrices(kind)
    S = SpinOrbitalADC(s.eps, s.nocc, 3, B=B)
    assert np.abs(sum(M.values()) - S.matrix(kind)).max() < 1e-12


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_matrix_adc2(pair, kind):
    F, s, B = pair
    M, _ = F.adc_matrices(kind)
    S = SpinOrbitalADC(s.eps, s.nocc, 2, B=B)
    assert np.abs(M[0] + M[1] + M[2] - S.matrix(kind)).max() < 1e-12


def test_amplitudes(pair):
    F, s, B = pair
    S = SpinOrbitalADC(s.eps, s.nocc, 3, B=B)
    assert np.abs(F.t2_tensor(1) - S.t2_1).max() < 1e-13
    assert np.abs(F.t2_tensor(2) - S.t2_2).max() < 1e-13
    assert np.abs(F.t1_tensor(2) - S.t1_2).max() < 1e-13
    assert abs(F.energy(2) - S.mp2_energy()) < 1e-13
    assert abs(F.energy(3) - S.mp3_energy()) < 1e-13
    # third-order singles (Eq. t_singles at k = 3): projection of the full
    # third-order effective Hamiltonian against the closed form with triples
    assert np.abs(F.t1_tensor(3)).max() > 1e-4
    assert np.abs(F.t1_tensor(3) - S.t1_3).max() < 1e-13


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_transition_second_order(pair, kind):
    F, s, B = pair
    T, bas = F.adc_transition(kind, 2)
    Tf = T[0] + T[1] + T[2]
    S = SpinOrbitalADC(s.eps, s.nocc, 3, B=B)
    one, two = S.basis_labels(kind)
    T1, T2 = S.ea_transition(2) if kind == "ea" else S.ip_transition(2)
    I = np.array(two)
    Ts = np.concatenate([T1, T2[:, I[:, 0], I[:, 1], I[:, 2]]], axis=1)
    assert np.abs(Tf - Ts).max() < 1e-13


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_transition_third_order(pair, kind):
    """T through k + l <= 3 (ADC(3)): the third-order piece alone and the sum."""
    F, s, B = pair
    T, bas = F.adc_transition(kind, 3)
    S = SpinOrbitalADC(s.eps, s.nocc, 3, B=B)
    one, two = S.basis_labels(kind)
    I = np.array(two)

    def flat(T1, T2):
        return np.concatenate([T1, T2[:, I[:, 0], I[:, 1], I[:, 2]]], axis=1)

    tr = S.ea_transition if kind == "ea" else S.ip_transition
    T3 = flat(*tr(3)) - flat(*tr(2))
    assert np.abs(T[3]).max() > 1e-4
    assert np.abs(T[3] - T3).max() < 1e-13
    assert np.abs(T[0] + T[1] + T[2] + T[3] - flat(*tr())).max() < 1e-13
