"""Unrestricted (open-shell) references in the spin-orbital oracles (UADC).

* Tier 1 (explicit spin-orbital equations) against tier 0 (operator
  definitions in Fock space) on open-shell references with nocc_a != nocc_b:
  amplitudes through t1(3), the EA/IP-ADC(2) and ADC(3) matrices and the
  transition moments, element by element.
* Restricted limit: an unrestricted reference built from one set of orbitals
  for both spins reproduces the restricted spectrum and MP energies.
"""
import numpy as np
import pytest

from adc_inputs import make_open_shell_system, make_system
from oracle.fock import ADCFock
from oracle.spinorb import SpinOrbitalADC
from oracle.unrestricted import unrestricted_spin_orbitals

OPEN = [(2, 1, 5, 10, 3), (3, 2, 5, 12, 4)]  # nocc_a, nocc_b, nmo, naux, seed


@pytest.fixture(scope="module", params=OPEN, ids=lambda c: f"a{c[0]}b{c[1]}n{c[2]}")
def open_pair(request):
    na, nb, nmo, naux, seed = request.param
    s = make_open_shell_system(na, nb, nmo, naux, seed=seed)
    eps, no, g = unrestricted_spin_orbitals(s.eps_a, s.eps_b, na, nb, 2.0 * s.B_a, 2.0 * s.B_b)
    return ADCFock.from_spin_orbitals(eps, no, g, 3), SpinOrbitalADC.from_spin_orbitals(eps, no, g, 3), (eps, no, g)


def test_open_shell_amplitudes(open_pair):
    F, S, _ = open_pair
    assert np.abs(F.t2_tensor(1) - S.t2_1).max() < 1e-13
    assert np.abs(F.t2_tensor(2) - S.t2_2).max() < 1e-13
    assert np.abs(F.t1_tensor(2) - S.t1_2).max() < 1e-13
    assert np.abs(F.t1_tensor(3)).max() > 1e-4
    assert np.abs(F.t1_tensor(3) - S.t1_3).max() < 1e-13
    assert abs(F.energy(2) - S.mp2_energy()) < 1e-13
    assert abs(F.energy(3) - S.mp3_energy()) < 1e-13


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_open_shell_matrices(open_pair, kind, order):
    F, _, (eps, no, g) = open_pair
    mats, _ = F.adc_matrices(kind)
    S = SpinOrbitalADC.from_spin_orbitals(eps, no, g, order)
    M = sum(mats[k] for k in range(order + 1))
    assert np.abs(M - S.matrix(kind)).max() < 1e-12
    assert np.abs(M - M.T).max() < 1e-12


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_open_shell_transition_moments(open_pair, kind):
    F, S, _ = open_pair
    T, _ = F.adc_transition(kind, 3)
    one, two = S.basis_labels(kind)
    I = np.array(two)
    tr = S.ea_transition if kind == "ea" else S.ip_transition
    for torder in (2, 3):
        T1, T2 = tr(torder)
        Ts = np.concatenate([T1, T2[:, I[:, 0], I[:, 1], I[:, 2]]], axis=1)
        assert np.abs(sum(T[k] for k in range(torder + 1)) - Ts).max() < 1e-13


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_restricted_limit(kind, order):
    s = make_system(3, 5, 14, seed=2)
    B = 2.0 * s.B
    R = SpinOrbitalADC(s.eps, 3, order, B=B)
    eps, no, g = unrestricted_spin_orbitals(s.eps, s.eps, 3, 3, B, B)
    U = SpinOrbitalADC.from_spin_orbitals(eps, no, g, order)
    wr = np.linalg.eigvalsh(R.matrix(kind))
    wu = np.linalg.eigvalsh(U.matrix(kind))
    assert np.abs(wr - wu).max() < 1e-11
    assert abs(R.mp2_energy() - U.mp2_energy()) < 1e-13
    if order == 3:
        assert abs(R.mp3_energy() - U.mp3_energy()) < 1e-13


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_matrix_free_sigma_matches_tier1(kind, order):
    """The matrix-free UADC sigma (two-particle block applied through the DF
    ladder of the per-spin factors) equals the tier-1 spin-orbital matrix."""
    from oracle.unrestricted import UnrestrictedADC

    s = make_open_shell_system(3, 2, 7, 20, seed=5)
    s.B_a *= 2.0
    s.B_b *= 2.0
    U = UnrestrictedADC(s, order, kind)
    eps, no, g = unrestricted_spin_orbitals(s.eps_a, s.eps_b, 3, 2, s.B_a, s.B_b)
    M = SpinOrbitalADC.from_spin_orbitals(eps, no, g, order).matrix(kind)
    assert U.dim == M.shape[0]
    assert np.abs(U.dense() - M).max() < 1e-12


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_davidson_on_unrestricted_sigma(kind):
    """The oracle Davidson (S = 1 for the spin-orbital basis) on the matrix-free
    UADC(3) sigma reproduces the lowest eigenvalues of its dense matrix."""
    from oracle.davidson import davidson
    from oracle.unrestricted import UnrestrictedADC

    s = make_open_shell_system(3, 2, 9, 24, seed=6)
    U = UnrestrictedADC(s, 3, kind)
    M = U.dense()
    w = np.linalg.eigvalsh(0.5 * (M + M.T))[:4]
    wd, _, _, _ = davidson(U, 4, tol=1e-10)
    assert np.abs(wd - w).max() < 1e-8


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_density_fitted_sigma_matches_tier1(kind, order):
    """The fully density-fitted UADC sigma (no v^3 or v^4 spin-orbital tensor:
    amplitudes through t1(3), one-particle block, and the EA coupling applied
    through B^Q) equals the tier-1 matrix; its amplitudes equal tier 1's."""
    from oracle.unrestricted import UnrestrictedDFADC

    s = make_open_shell_system(3, 2, 7, 20, seed=5)
    s.B_a *= 2.0
    s.B_b *= 2.0
    D = UnrestrictedDFADC(s, order, kind)
    eps, no, g = unrestricted_spin_orbitals(s.eps_a, s.eps_b, 3, 2, s.B_a, s.B_b)
    S = SpinOrbitalADC.from_spin_orbitals(eps, no, g, order)
    M = S.matrix(kind) * (1.0 if kind == "ea" else -1.0)  # IP: M_IP = -M_-
    assert D.dim == M.shape[0]
    assert np.abs(D.sigma(np.eye(D.dim)).T - M).max() < 1e-12 * max(1.0, np.abs(M).max())
    names = ("t2_1", "t1_2") + (("t2_2", "t1_3") if order == 3 else ())
    for name in names:
        assert np.abs(getattr(D, name) - getattr(S, name)).max() < 1e-14


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_density_fitted_davidson_larger(kind):
    """At a size the dense tier-1 matrix would not reach (EA dim ~ 2.6e4), the DF
    sigma drives the oracle Davidson to converged UADC(3) roots."""
    from oracle.davidson import davidson
    from oracle.unrestricted import UnrestrictedDFADC

    s = make_open_shell_system(6, 5, 40, 60, seed=7)
    D = UnrestrictedDFADC(s, 3, kind)
    w, Y, it, ns = davidson(D, 3, tol=1e-9, res_tol=1e-6)
    R = D.sigma(Y) - w[:, None] * Y
    assert np.abs(np.linalg.norm(R, axis=1)).max() < 1e-5
    assert np.all(np.diff(w) >= -1e-12)


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_open_shell_koopmans_limit(kind):
    """B -> 0: the UADC(3) roots approach the orbital energies (EA: the lowest
    virtual spin orbitals; IP: minus the highest occupied ones) with spectroscopic
    factor 1 each (one spin-orbital component)."""
    from oracle.davidson import dense_roots
    from oracle.unrestricted import UnrestrictedDFADC, spin_orbital_df

    s = make_open_shell_system(3, 2, 6, 12, seed=8)
    s.B_a *= 1e-4
    s.B_b *= 1e-4
    D = UnrestrictedDFADC(s, 3, kind)
    eps, no, _ = spin_orbital_df(s)
    ref = np.sort(eps[no:])[:2] if kind == "ea" else np.sort(-eps[:no])[:2]
    w, Y = dense_roots(D, 2)
    assert np.abs(w - ref).max() < 1e-6
    assert np.abs(D.spectroscopic_factors(Y) - 1.0).max() < 1e-6


def test_spectroscopic_factors_match_tier1():
    from oracle.unrestricted import UnrestrictedDFADC

    s = make_open_shell_system(3, 2, 7, 20, seed=5)
    D = UnrestrictedDFADC(s, 3, "ea")
    eps, no, g = unrestricted_spin_orbitals(s.eps_a, s.eps_b, 3, 2, s.B_a, s.B_b)
    S = SpinOrbitalADC.from_spin_orbitals(eps, no, g, 3)
    T1, T2 = S.ea_transition()
    _, two = S.basis_labels("ea")
    I = np.array(two)
    T = np.concatenate([T1, T2[:, I[:, 0], I[:, 1], I[:, 2]]], axis=1)
    Y = np.random.default_rng(1).standard_normal((3, D.dim))
    Yn = Y / np.linalg.norm(Y, axis=1)[:, None]
    assert np.abs(D.spectroscopic_factors(Y) - ((Yn @ T.T) ** 2).sum(axis=1)).max() < 1e-13
