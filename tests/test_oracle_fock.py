"""Pins of the tier-0 (Fock-space) oracle against facts that do not come from it.

* Koopmans limit: the zeroth-order matrices are diagonal with eps_a (EA 1p),
  eps_a + eps_b - eps_i (EA 2p1h), eps_i and eps_i + eps_j - eps_a (IP, paper's
  M_- sign) -- Sec. II A with H~(0) = H(0).
* The second-order ground-state energy equals the closed-form MP2 energy
  (the amplitudes are MP-equivalent, Sec. II A after Eq. t_doubles).
* M is Hermitian at every order (Eqs. M_ea, M_ip).
* ADC(n) main-state energies agree with exact full-CI electron attachment /
  ionisation energies through order n: scaling B by lam scales V by lam^2,
  so the error must fall as lam^(2(n+1)) (lam^6 for ADC(2), lam^8 for ADC(3)).
* T^(0) is the unit matrix on the 1p / 1h columns (Eqs. T_ea, T_ip).
"""
import numpy as np
import pytest

from adc_inputs import make_system
from oracle.fock import ADCFock


@pytest.fixture(scope="module")
def tiny():
    s = make_system(2, 3, 10, seed=5)
    return s, ADCFock(s.eps, 2, 3, B=2.0 * s.B)


def test_koopmans_order0(tiny):
    s, F = tiny
    e = F.eps_so
    for kind in ("ea", "ip"):
        P, bas, orders = F.adc_pieces(kind)
        D = P[0]
        assert np.abs(D - np.diag(np.diag(D))).max() < 1e-13
        for k, (lab, o, _) in enumerate(bas):
            if lab[0] == "p":
                ref = e[lab[1]]
            elif lab[0] == "pph":
                ref = e[lab[2]] + e[lab[3]] - e[lab[1]]
            elif lab[0] == "h":
                ref = e[lab[1]]
            else:
                ref = e[lab[1]] + e[lab[2]] - e[lab[3]]
            assert abs(D[k, k] - ref) < 1e-13


def test_mp2_closed_form(tiny):
    s, F = tiny
    B = 2.0 * s.B
    eri = np.einsum("Qpq,Qrs->pqrs", B, B)
    no = s.nocc
    eo, ev = s.eps[:no], s.eps[no:]
    ovov = eri[:no, no:, :no, no:]
    D = eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] - ev[None, None, None, :]
    emp2 = np.sum(ovov * (2 * ovov - ovov.transpose(0, 3, 2, 1)) / D)
    assert abs(F.energy(2) - emp2) < 1e-14
    assert abs(F.energy(1)) < 1e-14


def test_hermitian(tiny):
    s, F = tiny
    for kind in ("ea", "ip"):
        M, _ = F.adc_matrices(kind)
        for n, m in M.items():
            assert np.abs(m - m.T).max() < 1e-13


def test_transition_order0(tiny):
    s, F = tiny
    for kind in ("ea", "ip"):
        T, bas = F.adc_transition(kind, 0)
        for k, (lab, o, _) in enumerate(bas):
            col = T[0][:, k]
            if o == 0:
                ref = np.zeros(F.nso)
                ref[lab[1]] = 1.0
                assert np.abs(col - ref).max() < 1e-14
            else:
                assert np.abs(col).max() < 1e-14


@pytest.mark.parametrize("kind", ["ea", "ip"])
@pytest.mark.parametrize("order", [2, 3])
def test_exact_through_order_n(kind, order):
    s = make_system(2, 3, 10, seed=5)
    errs = []
    for lam in (0.5, 0.25):
        F = ADCFock(s.eps, 2, order, B=lam * s.B)
        M, _ = F.adc_matrices(kind)
        w = np.linalg.eigvalsh(sum(M.values()))
        H = {n: F.H0[n] + F.V[n] for n in F.sectors}
        E0 = np.linalg.eigvalsh(H[F.N])[0]
        if kind == "ea":
            errs.append(abs(w[0] - (np.linalg.eigvalsh(H[F.N + 1])[0] - E0)))
        else:
            errs.append(abs(w[-1] - (E0 - np.linalg.eigvalsh(H[F.N - 1])[0])))
    slope = np.log2(errs[0] / errs[1])
    assert slope > 2 * (order + 1) - 0.3, (errs, slope)
