"""Unrestricted (open-shell) references for the spin-orbital oracles.
TEST INFRASTRUCTURE ONLY -- nothing in the GPU product path may import this.

The paper runs EA/IP-UADC(n) for open-shell molecules (Sec. II; the TEMPO
radical, Sec. IV): the working equations are the spin-orbital ones, with
alpha and beta orbitals that differ.  Here the spin-orbital energies and
antisymmetrised integrals of such a reference are built from per-spin
orbital energies and per-spin DF factors, with the two-electron integrals
(p_s q_s | r_t s_t) = sum_Q B^Q_{s,pq} B^Q_{t,rs} (Eq. 19 for each spin
pair) and <PQ||RS> = (PR|QS) d(s_P,s_R) d(s_Q,s_S) - (PS|QR) d(s_P,s_S) d(s_Q,s_R).

Spin-orbital order: occupied alpha, occupied beta, virtual alpha, virtual beta
(so the first nocc_a + nocc_b spin orbitals are the occupied ones, as the
tier-0 and tier-1 oracles expect).
"""
from __future__ import annotations

import numpy as np


def spin_orbital_order(nmo, nocc_a, nocc_b):
    """(spin [nso], spatial index [nso]) of each spin orbital in the order above."""
    spin = np.concatenate([np.zeros(nocc_a), np.ones(nocc_b), np.zeros(nmo - nocc_a), np.ones(nmo - nocc_b)]).astype(int)
    idx = np.concatenate([np.arange(nocc_a), np.arange(nocc_b), np.arange(nocc_a, nmo), np.arange(nocc_b, nmo)])
    return spin, idx


def unrestricted_spin_orbitals(eps_a, eps_b, nocc_a, nocc_b, B_a, B_b):
    """(eps_so [nso], no, <PQ||RS> [nso]^4) of an unrestricted reference."""
    nmo = len(eps_a)
    spin, idx = spin_orbital_order(nmo, nocc_a, nocc_b)
    eps = np.where(spin == 0, np.asarray(eps_a)[idx], np.asarray(eps_b)[idx])
    B = np.stack([np.asarray(B_a, dtype=float), np.asarray(B_b, dtype=float)])  # [spin, Q, p, q]
    # chemists' (PR|QS) over spin orbitals with the spin of each pair: B^Q_{s_P, p r} B^Q_{s_Q, q s}
    Bso = B[spin[:, None], :, idx[:, None], idx[None, :]]  # [P, R, Q]: B^Q_{s_P, p r}, valid where s_P = s_R
    same = (spin[:, None] == spin[None, :])
    Bso = Bso * same[:, :, None]
    chem = np.einsum("PRQ,XSQ->PRXS", Bso, Bso)  # (PR|XS)
    phys = chem.transpose(0, 2, 1, 3)  # <PX|RS> = (PR|XS)
    return eps, nocc_a + nocc_b, phys - phys.transpose(0, 1, 3, 2)


class UnrestrictedADC:
    """Matrix-free EA/IP-UADC(n) sigma = M Y on the spin-orbital basis of the
    tier-1 oracle (EA: 1p a, 2p1h (i, a<b); IP: 1h i, 2h1p (i<j, a); the IP
    matrix is the paper's M_-).

    The one-particle and coupling blocks come from the tier-1 equations.  The
    two-particle block is applied without forming it: its zeroth-order part is
    diagonal, and its first-order part (ADC(3)) is, for EA,
      sum_cd <ab||cd> Y_icd / 2 = sum_Q (B^Q_v Y_i B^Q_v)_ab
    (the DF ladder, Eq. 19, with the spin-block-diagonal virtual factor: its
    alpha-alpha, beta-beta and alpha-beta blocks are the three unrestricted
    ladders), minus the ring terms sum_jc <aj||ci> Y_jcb - (a <-> b); for IP
    -1/2 sum_kl <ij||kl> Y_kla plus the ring terms sum_kb <ka||ib> Y_kjb - (i <-> j).
    """

    def __init__(self, sysm, order=3, kind="ea"):
        from oracle.spinorb import SpinOrbitalADC

        assert order in (2, 3) and kind in ("ea", "ip")
        na, nb = sysm.nocc_a, sysm.nocc_b
        eps, no, g = unrestricted_spin_orbitals(sysm.eps_a, sysm.eps_b, na, nb, sysm.B_a, sysm.B_b)
        self.order, self.kind = order, kind
        self.so = S = SpinOrbitalADC.from_spin_orbitals(eps, no, g, order)
        self.no, self.nv = S.no, S.nv
        spin, idx = spin_orbital_order(sysm.nmo, na, nb)
        B = np.stack([np.asarray(sysm.B_a, dtype=float), np.asarray(sysm.B_b, dtype=float)])
        sv, iv = spin[no:], idx[no:]
        self.Bv = B[sv[:, None], :, iv[:, None], iv[None, :]].transpose(2, 0, 1) * (sv[:, None] == sv[None, :])
        if kind == "ea":
            self.M11, self.M12 = S.ea_m11(), S.ea_m12()
        else:
            self.M11, self.M12 = S.ip_m11(), S.ip_m12()
        one, two = S.basis_labels(kind)
        self.n1 = len(one)
        self.I = np.array(two).T
        self.dim = self.n1 + self.I.shape[1]

    def _full(self, y2):
        """Restricted-pair amplitudes -> tensor antisymmetric in the like pair."""
        n = y2.shape[0]
        i0, i1, i2 = self.I
        if self.kind == "ea":
            F = np.zeros((n, self.no, self.nv, self.nv))
            F[:, i0, i1, i2] = y2
            F[:, i0, i2, i1] = -y2
        else:
            F = np.zeros((n, self.no, self.no, self.nv))
            F[:, i0, i1, i2] = y2
            F[:, i1, i0, i2] = -y2
        return F

    def sigma(self, Y):
        Y = np.atleast_2d(np.asarray(Y, dtype=float))
        y1, F = Y[:, : self.n1], self._full(Y[:, self.n1 :])
        S = self.so
        s1 = y1 @ self.M11.T + 0.5 * np.einsum("pjcd,njcd->np", self.M12, F)
        S2 = np.einsum("pjcd,np->njcd", self.M12, y1)
        if self.kind == "ea":
            S2 += (S.ev[None, None, :, None] + S.ev[None, None, None, :] - S.eo[None, :, None, None]) * F
            if self.order >= 3:
                for BQ in self.Bv:
                    S2 += BQ @ F @ BQ
                R = np.einsum("ajci,njcb->niab", S.blk("vovo"), F)
                S2 -= R - R.transpose(0, 1, 3, 2)
        else:
            S2 += (S.eo[None, :, None, None] + S.eo[None, None, :, None] - S.ev[None, None, None, :]) * F
            if self.order >= 3:
                S2 -= 0.5 * np.einsum("ijkl,nkla->nija", S.blk("oooo"), F)
                R = np.einsum("kaib,nkjb->nija", S.blk("ovov"), F)
                S2 += R - R.transpose(0, 2, 1, 3)
        i0, i1, i2 = self.I
        return np.concatenate([s1, S2[:, i0, i1, i2]], axis=1)

    def dense(self):
        return self.sigma(np.eye(self.dim)).T

    # the spin-orbital basis is orthonormal: metric S = 1 (for the oracle Davidson)
    def apply_S(self, Y):
        return np.array(Y, dtype=float)

    def solve_S(self, Y):
        return np.array(Y, dtype=float)

    def diagonal(self):
        """diag(M_11) and the zeroth-order two-particle energies (Davidson preconditioner)."""
        S = self.so
        i0, i1, i2 = self.I
        if self.kind == "ea":
            d2 = S.ev[i1] + S.ev[i2] - S.eo[i0]
        else:
            d2 = S.eo[i0] + S.eo[i1] - S.ev[i2]
        return np.concatenate([np.diag(self.M11), d2])
