"""Tier-2 (spin-adapted, density-fitted) oracle against tier 1 and against
facts that hold independently of both.

* sigma_SA = S^-1 E^T M_SO E Y for the doublet embedding E (Sec. III B), EA and
  IP, ADC(2) and ADC(3); S M_SA is symmetric; S = E^T E.
* Density fitting with a complete auxiliary set reproduces the four-index
  result exactly (Eq. 19): B is the exact factor of a random positive
  semi-definite (pq|rs).
* Spectroscopic factors with the Appendix normalisation equal twice the
  spin-orbital factor of one M_S component (Eq. spec_factors); in the
  Koopmans limit (B -> 0) the roots approach eps_a / -eps_i with P -> 2.
* The oracle Davidson iteration reproduces the dense solution.
"""
import numpy as np
import pytest

from adc_inputs import make_psd_eri, make_system
from oracle.davidson import davidson, dense_roots, spectroscopic_factors
from oracle.spinadapted import SpinAdaptedADC, embedding
from oracle.spinorb import SpinOrbitalADC


def _sa_from_so(S, kind, o, v):
    E = embedding(o, v, kind)
    M = S.matrix(kind) * (1.0 if kind == "ea" else -1.0)
    Sm = E.T @ E
    return np.linalg.solve(Sm, E.T @ M @ E), Sm


@pytest.mark.parametrize("o,v,seed", [(3, 4, 2), (4, 3, 3), (2, 5, 4)])
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_sigma_matches_spin_orbital(o, v, seed, order, kind):
    s = make_system(o, v, 16, seed=seed)
    B = 2.0 * s.B
    T = SpinAdaptedADC(s.eps, o, B, order, kind)
    Msa, Sm = _sa_from_so(SpinOrbitalADC(s.eps, o, order, B=B), kind, o, v)
    D = T.dense()
    assert np.abs(D - Msa).max() < 1e-12
    assert np.abs(T.apply_S(np.eye(T.dim)) - Sm).max() < 1e-15
    A = T.apply_S(D.T).T
    assert np.abs(A - A.T).max() < 1e-12


@pytest.mark.parametrize("o,v,seed", [(3, 4, 2), (2, 5, 4)])
def test_third_order_singles_match_spin_orbital(o, v, seed):
    """Spatial t_i^a(3) equals the alpha-alpha block of the spin-orbital one
    (spin orbital 2p + s); the alpha-beta block vanishes."""
    s = make_system(o, v, 16, seed=seed)
    B = 2.0 * s.B
    T = SpinAdaptedADC(s.eps, o, B, 3, "ea")
    S = SpinOrbitalADC(s.eps, o, 3, B=B)
    assert np.abs(S.t1_3[0::2, 1::2]).max() == 0.0
    assert np.abs(T.t1_3).max() > 1e-4
    assert np.abs(T.t1_3 - S.t1_3[0::2, 0::2]).max() < 1e-14
    assert np.abs(T.t1_3 - S.t1_3[1::2, 1::2]).max() < 1e-14


def test_mp_energies_match_spin_orbital():
    s = make_system(3, 5, 16, seed=2)
    B = 2.0 * s.B
    S = SpinOrbitalADC(s.eps, 3, 3, B=B)
    e2 = SpinAdaptedADC(s.eps, 3, B, 2, "ea").mp_energies()
    e3 = SpinAdaptedADC(s.eps, 3, B, 3, "ip").mp_energies()
    assert len(e2) == 1 and len(e3) == 2
    assert abs(e2[0] - S.mp2_energy()) < 1e-14 and abs(e3[0] - e2[0]) < 1e-15
    assert abs(e3[1] - S.mp3_energy()) < 1e-14


@pytest.mark.parametrize("order,torder", [(2, None), (3, None), (3, 2)])
@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_transition_moments_match_spin_orbital(order, torder, kind):
    """X = T E Y~ for every S-normalised vector: the spatial T (through order n,
    or second order for ADC(3) on request) acting on a doublet vector equals the
    spin-orbital T on its embedding (P summed over both spin components)."""
    o, v = 3, 4
    s = make_system(o, v, 16, seed=6)
    B = 2.0 * s.B
    T = SpinAdaptedADC(s.eps, o, B, order, kind)
    S = SpinOrbitalADC(s.eps, o, order, B=B)
    E = embedding(o, v, kind)
    T1, T2 = S.ea_transition(torder) if kind == "ea" else S.ip_transition(torder)
    _, two = S.basis_labels(kind)
    I = np.array(two)
    Tso = np.concatenate([T1, T2[:, I[:, 0], I[:, 1], I[:, 2]]], axis=1)
    Y = np.random.default_rng(0).standard_normal((5, T.dim))
    P = spectroscopic_factors(T, Y, torder)
    for r in range(5):
        u = E @ Y[r]
        u /= np.linalg.norm(u)
        assert abs(P[r] - 2.0 * np.sum((Tso @ u) ** 2)) < 1e-12


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_df_complete_auxiliary_set(kind):
    o, v = 2, 4
    nmo = o + v
    eri = make_psd_eri(nmo, seed=9, scale=0.4)
    # exact factorisation over the pair space: (pq|rs) = sum_Q B^Q_pq B^Q_rs
    G = eri.reshape(nmo * nmo, nmo * nmo)
    lam, U = np.linalg.eigh(0.5 * (G + G.T))
    keep = lam > 1e-12 * lam.max()
    B = (U[:, keep] * np.sqrt(lam[keep])).T.reshape(-1, nmo, nmo)
    assert B.shape[0] <= nmo * (nmo + 1) // 2
    eps = make_system(o, v, 4, seed=1).eps
    T = SpinAdaptedADC(eps, o, B, 3, kind)
    S = SpinOrbitalADC(eps, o, 3, eri=eri)
    Msa, _ = _sa_from_so(S, kind, o, v)
    assert np.abs(T.dense() - Msa).max() < 1e-12
    # the DF forms of t1(3) and of the MP energies reproduce the four-index ones
    assert np.abs(T.t1_3 - S.t1_3[0::2, 0::2]).max() < 1e-13
    assert abs(T.mp_energies()[0] - S.mp2_energy()) < 1e-13
    assert abs(T.mp_energies()[1] - S.mp3_energy()) < 1e-13


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_eigenvalues_and_spectroscopic_factors(kind):
    o, v = 3, 4
    s = make_system(o, v, 16, seed=4)
    B = 2.0 * s.B
    T = SpinAdaptedADC(s.eps, o, B, 3, kind)
    S = SpinOrbitalADC(s.eps, o, 3, B=B)
    w, Y = dense_roots(T, 4)
    M = S.matrix(kind) * (1.0 if kind == "ea" else -1.0)
    wso = np.linalg.eigvalsh(M)
    for x in w:
        assert np.min(np.abs(wso - x)) < 1e-11
    E = embedding(o, v, kind)
    T1, T2 = S.ea_transition() if kind == "ea" else S.ip_transition()
    _, two = S.basis_labels(kind)
    I = np.array(two)
    Tso = np.concatenate([T1, T2[:, I[:, 0], I[:, 1], I[:, 2]]], axis=1)
    P = spectroscopic_factors(T, Y)
    for r in range(4):
        u = E @ Y[r]
        u /= np.linalg.norm(u)
        assert abs(P[r] - 2.0 * np.sum((Tso @ u) ** 2)) < 1e-12


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_koopmans_limit(kind):
    s = make_system(3, 6, 12, seed=7)
    T = SpinAdaptedADC(s.eps, 3, 1e-4 * s.B, 3, kind)
    w, Y = dense_roots(T, 2)
    ref = s.eps[3:5] if kind == "ea" else -s.eps[2:0:-1]
    assert np.abs(w - ref).max() < 1e-6
    assert np.abs(spectroscopic_factors(T, Y) - 2.0).max() < 1e-6


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_davidson_matches_dense(kind):
    s = make_system(4, 12, 40, seed=0)
    T = SpinAdaptedADC(s.eps, 4, s.B, 3, kind)
    w, _ = dense_roots(T, 4)
    wd, Yd, it, ns = davidson(T, 4, tol=1e-10)
    assert np.abs(w - wd).max() < 1e-9
