"""Symmetries the memory-lean setup relies on, checked on the oracle's own amplitudes.

* t_ij^ab = t_ji^ba for t2(1) and t2(2) (closed-shell amplitudes, Eqs. t_doubles), so the ladder
  L_ij = sum_Q B^Q t_ij B^Q of a symmetric B^Q (Eq. 19) satisfies L_ji = L_ij^T: the lean setup
  evaluates the pairs i <= j only.
* A contraction with tau = 2 t - t(ab swap) equals twice the contraction with t minus the one
  with the virtual pair of t swapped, and (ia|jc) ring2 = 2 (ia|jc) - (ji|ac): the lean sigma
  holds neither tau nor ring2 and forms these terms from t and the integrals.
"""
import numpy as np

from adc_inputs import make_system
from oracle.spinadapted import SpinAdaptedADC, df_ladder


def test_amplitude_pair_symmetry_and_ladder_transpose():
    o, v, naux = 4, 11, 23
    s = make_system(o, v, naux, seed=7)
    T = SpinAdaptedADC(s.eps, o, s.B, 3, "ea")
    for t in (T.t, T.t_2):
        assert np.abs(t - t.transpose(1, 0, 3, 2)).max() <= 1e-14 * np.abs(t).max()
    Bvv = s.B[:, o:, o:]
    for i in range(o):
        for j in range(o):
            Lij = df_ladder(Bvv, T.t[i, j])
            Lji = df_ladder(Bvv, T.t[j, i])
            assert np.abs(Lji - Lij.T).max() <= 1e-13 * np.abs(Lij).max()


def test_tau_and_ring_expansions():
    o, v, naux = 3, 9, 17
    s = make_system(o, v, naux, seed=8)
    T = SpinAdaptedADC(s.eps, o, s.B, 3, "ea")
    t = T.t
    tau = 2.0 * t - t.transpose(0, 1, 3, 2)
    Y = np.random.default_rng(9).standard_normal((o, v, v))
    a = np.einsum("jmce,jcd->med", tau, Y)
    b = 2.0 * np.einsum("jmce,jcd->med", t, Y) - np.einsum("jmec,jcd->med", t, Y)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
    Bov, Boo, Bvv = s.B[:, :o, o:], s.B[:, :o, :o], s.B[:, o:, o:]
    ovov = np.einsum("Qia,Qjc->iajc", Bov, Bov)
    oovv = np.einsum("Qji,Qac->jiac", Boo, Bvv)
    ring2 = 2.0 * ovov - oovv.transpose(1, 2, 0, 3)
    a = np.einsum("iajc,jcb->iab", ring2, Y)
    b = 2.0 * np.einsum("iajc,jcb->iab", ovov, Y) - np.einsum("jiac,jcb->iab", oovv, Y)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
