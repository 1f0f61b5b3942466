"""Tier-1 oracle: explicit spin-orbital EA/IP-ADC(n) working equations (n = 2, 3).
TEST INFRASTRUCTURE ONLY -- nothing in the GPU product path may import this.

The paper defers its spin-orbital working equations to earlier work; the
equations below were derived here from the definitions it states (Eqs. M_ea,
M_ip, T_ea, T_ip with the BCH series Eqs. H_bch, ap_bch and the amplitude
conditions Eqs. t_singles, t_doubles).  For a diagonal Fock operator the EA
1p-1p block is the virtual-virtual one-body part of the effective Hamiltonian,
the coupling block is its two-body (vo|vv) part and the 2p1h block its zeroth-
and first-order parts between 2p1h determinants; the IP blocks are the
particle-hole analogues.  Every block, order by order, is checked element by
element against the brute-force Fock-space evaluation (``fock.py``) on random
tiny systems.

Notation (spin orbitals, occupied i,j,k,l,m and virtual a,b,c,d,e):
  g[pqrs] = <pq||rs>,  D_ij^ab = e_i + e_j - e_a - e_b,  D_i^a = e_i - e_a
  t_ij^ab(1) = <ab||ij> / D_ij^ab
  t_ij^ab(2) = [ 1/2 <ab||cd> t_ij^cd + 1/2 <kl||ij> t_kl^ab
                 + P(ij)P(ab) <kb||cj> t_ik^ac ] / D_ij^ab
  t_i^a(2)   = [ -1/2 <ka||cd> t_ik^cd - 1/2 <kl||ic> t_kl^ac ] / D_i^a
  (t1(1) = 0 because the Fock operator is diagonal.)
  t_i^a(3)   = [ <aj||ib> t_j^b(2) - 1/2 <ka||cd> t_ik^cd(2) - 1/2 <kl||ic> t_kl^ac(2)
                 + 1/4 t_jk^bc W_ijk^abc ] / D_i^a + 1/2 t_ij^ab t_j^b(2)
  with the connected first-order triples
  W_ijk^abc = P(k/ij) P(a/bc) <bc||dk> t_ij^ad - P(i/jk) P(c/ab) <lc||jk> t_il^ab.
  This is the singles projection (Eq. t_singles) of the third-order effective
  Hamiltonian: [V, sigma2] gives the CC-like singles terms of t1(2) and t2(2)
  plus t1(2)+ V; the double commutators with H0 turn into -1/2 t1(2)+ V and
  -1/2 (D t1(2))+ t2(1), which with it leave 1/2 t_ij^ab t_j^b(2); and
  1/2 [[V, sigma1], sigma1] leaves the triples term T2+ V T2.

Basis conventions (identical to fock.py): EA 2p1h state (i,a,b) is
a_b+ a_a+ a_i |Phi>; IP 2h1p state (i,j,a) is (a_a+ a_j a_i)+ acting on the
ket side, i.e. the paper's h operators.  Six-index blocks are stored for all
index values, antisymmetric in the like pair; the restricted basis keeps a<b
(EA) or i<j (IP).  The IP matrix is the paper's M_- (eigenvalues E_N - E_{N-1}).
"""
from __future__ import annotations

from itertools import combinations

import numpy as np


def antisym_integrals(eri_spatial: np.ndarray) -> np.ndarray:
    """<PQ||RS> for P = 2p + s from chemists' (pq|rs) (Sec. III B spin integration)."""
    nmo = eri_spatial.shape[0]
    nso = 2 * nmo
    spin = np.arange(nso) % 2
    sp = np.arange(nso) // 2
    phys = eri_spatial[sp[:, None, None, None], sp[None, None, :, None], sp[None, :, None, None], sp[None, None, None, :]]
    same = (spin[:, None, None, None] == spin[None, None, :, None]) & (spin[None, :, None, None] == spin[None, None, None, :])
    phys = phys * same
    return phys - phys.transpose(0, 1, 3, 2)


def _anti_ab(X):
    """X - X(a<->b) for the last two axes of a 3-index-pair tensor."""
    return X - np.swapaxes(X, -1, -2)


class SpinOrbitalADC:
    """Dense spin-orbital EA/IP-ADC(order) for small systems."""

    def __init__(self, eps, nocc, order, B=None, eri=None):
        eps = np.asarray(eps, dtype=float)
        if eri is None:
            eri = np.einsum("Qpq,Qrs->pqrs", B, B)
        self._init_spin_orbitals(np.repeat(eps, 2), 2 * nocc, antisym_integrals(np.asarray(eri, dtype=float)), order)

    @classmethod
    def from_spin_orbitals(cls, eps_so, no, g, order):
        """Any reference given in spin orbitals (eps_so [nso], the first `no`
        occupied, g = <PQ||RS>): the same working equations serve the
        unrestricted open-shell case (UADC, Sec. II)."""
        self = cls.__new__(cls)
        self._init_spin_orbitals(np.asarray(eps_so, dtype=float), no, np.asarray(g, dtype=float), order)
        return self

    def _init_spin_orbitals(self, e, no, g, order):
        self.order = order
        self.no = no
        self.nso = len(e)
        self.nv = self.nso - self.no
        o, v = slice(0, self.no), slice(self.no, self.nso)
        self._sl = {"o": o, "v": v}
        self.g = g
        self.eo, self.ev = e[o], e[v]
        self.D2 = self.eo[:, None, None, None] + self.eo[None, :, None, None] - self.ev[None, None, :, None] - self.ev[None, None, None, :]
        self.D1 = self.eo[:, None] - self.ev[None, :]
        self._amplitudes()

    def blk(self, s):
        sl = self._sl
        return self.g[sl[s[0]], sl[s[1]], sl[s[2]], sl[s[3]]]

    # ---- amplitudes (Eqs. t_singles, t_doubles; MP-equivalent) ----------
    def _amplitudes(self):
        g = self.blk
        t = g("vvoo").transpose(2, 3, 0, 1) / self.D2
        self.t2_1 = t
        X = np.einsum("kbcj,ikac->ijab", g("ovvo"), t)
        ring = X - X.transpose(1, 0, 2, 3) - X.transpose(0, 1, 3, 2) + X.transpose(1, 0, 3, 2)
        num = 0.5 * np.einsum("abcd,ijcd->ijab", g("vvvv"), t) + 0.5 * np.einsum("klij,klab->ijab", g("oooo"), t) + ring
        self.t2_2 = num / self.D2
        num1 = -0.5 * np.einsum("kacd,ikcd->ia", g("ovvv"), t) - 0.5 * np.einsum("klic,klac->ia", g("ooov"), t)
        self.t1_2 = num1 / self.D1
        if self.order >= 3:
            self.t1_3 = self._t1_third_order()

    def _t1_third_order(self):
        """t_i^a(3) of the module docstring, with the triples term expanded.

        1/4 t_jk^bc W_ijk^abc is summed permutation by permutation; equal
        terms are collected, which leaves four particle contractions (E1..E4)
        and four hole contractions (F1..F4), none of them forming W.
        """
        g = self.blk
        t, t1, t2 = self.t2_1, self.t1_2, self.t2_2
        A = np.einsum("ajib,jb->ia", g("voov"), t1)
        A -= 0.5 * np.einsum("kacd,ikcd->ia", g("ovvv"), t2) + 0.5 * np.einsum("klic,klac->ia", g("ooov"), t2)
        vvvo, ovoo = g("vvvo"), g("ovoo")
        E1 = np.einsum("ijad,jkbc,bcdk->ia", t, t, vvvo, optimize=True)  # P(k/ij): 1, (jk)
        E2 = np.einsum("jkad,jkbc,bcdi->ia", t, t, vvvo, optimize=True)  # (ik)
        E3 = -np.einsum("acdk,ijbd,jkbc->ia", vvvo, t, t, optimize=True)  # P(a/bc): (ab), (ac)
        E4 = -np.einsum("acdi,jkbc,jkbd->ia", vvvo, t, t, optimize=True)  # (ik)(ab), (ik)(ac)
        F1 = np.einsum("ilab,jkbc,lcjk->ia", t, t, ovoo, optimize=True)  # P(c/ab): 1, (bc)
        F2 = -np.einsum("lcik,jkbc,jlab->ia", ovoo, t, t, optimize=True)  # P(i/jk): (ij), (ik)
        F3 = np.einsum("lajk,jkbc,ilbc->ia", ovoo, t, t, optimize=True)  # (ac)
        F4 = -np.einsum("laik,jkbc,jlbc->ia", ovoo, t, t, optimize=True)  # (ij)(ac), (ik)(ac)
        W = 0.25 * (2 * E1 + E2 + 4 * E3 + 2 * E4) - 0.25 * (2 * F1 + 4 * F2 + F3 + 2 * F4)
        return (A + W) / self.D1 + 0.5 * np.einsum("ijab,jb->ia", t, t1)

    def mp2_energy(self):
        return 0.25 * float(np.einsum("ijab,ijab->", self.blk("oovv"), self.t2_1))

    def mp3_energy(self):
        """Third-order energy <Phi|H~(3)|Phi> = 1/4 sum <ij||ab> t_ij^ab(2) (Sec. III A step 2)."""
        return 0.25 * float(np.einsum("ijab,ijab->", self.blk("oovv"), self.t2_2))

    # ---- EA blocks ---------------------------------------------------------
    def ea_m11(self):
        """1p-1p block M_ab through order n (one-body vv part of the effective H)."""
        g = self.blk
        t = self.t2_1
        M = np.diag(self.ev).copy()
        X = np.einsum("klac,klbc->ab", t, g("oovv"))
        M -= 0.25 * (X + X.T)
        if self.order >= 3:
            t1, t2 = self.t1_2, self.t2_2
            X = np.einsum("kc,kacb->ab", t1, g("ovvv"))
            M += X + X.T
            X = np.einsum("klac,klbc->ab", t2, g("oovv"))
            M -= 0.25 * (X + X.T)
            X = np.einsum("klac,bcde,klde->ab", t, g("vvvv"), t)
            M -= 0.125 * (X + X.T)
            M += 0.5 * np.einsum("acbd,klce,klde->ab", g("vvvv"), t, t)
            X = np.einsum("kmac,kdlb,lmcd->ab", t, g("ovov"), t)
            M -= 0.5 * (X + X.T)
            M -= 0.5 * np.einsum("kalb,kmcd,lmcd->ab", g("ovov"), t, t)
        return M

    def ea_m12(self):
        """Coupling block M[a, j, c, d] (1p row, 2p1h column) through order n-1."""
        g = self.blk
        M = -g("vovv").copy()
        if self.order >= 3:
            t = self.t2_1
            M -= 0.5 * np.einsum("ajlm,lmcd->ajcd", g("vooo"), t)
            X = np.einsum("aecm,jmde->ajcd", g("vvvo"), t)
            M -= X - X.transpose(0, 1, 3, 2)
        return M

    def ea_m22(self):
        """2p1h-2p1h block M[i,a,b, j,c,d] through order n-2."""
        no, nv = self.no, self.nv
        I, J = np.eye(no), np.eye(nv)
        d = self.ev[:, None] + self.ev[None, :]
        M = np.einsum("ij,ac,bd->iabjcd", I, J, J) * (d[None, :, :, None, None, None] - self.eo[:, None, None, None, None, None])
        M = M - M.transpose(0, 1, 2, 3, 5, 4)
        if self.order >= 3:
            M = M + np.einsum("ij,abcd->iabjcd", I, self.blk("vvvv"))
            R = np.einsum("bd,ajci->iabjcd", J, self.blk("vovo"))
            R = R - R.transpose(0, 2, 1, 3, 4, 5)
            M = M - (R - R.transpose(0, 1, 2, 3, 5, 4))
        return M

    # ---- IP blocks ---------------------------------------------------------
    def ip_m11(self):
        """1h-1h block M_ij (paper's M_- convention) through order n."""
        g = self.blk
        t = self.t2_1
        M = np.diag(self.eo).copy()
        X = np.einsum("ilcd,jlcd->ij", t, g("oovv"))
        M += 0.25 * (X + X.T)
        if self.order >= 3:
            t1, t2 = self.t1_2, self.t2_2
            X = np.einsum("kc,cikj->ij", t1, g("vooo"))
            M += X + X.T
            X = np.einsum("ikcd,cdjk->ij", t2, g("vvoo"))
            M += 0.25 * (X + X.T)
            X = np.einsum("ikcd,jklm,lmcd->ij", t, g("oooo"), t)
            M += 0.125 * (X + X.T)
            M -= 0.5 * np.einsum("ikjl,kmcd,lmcd->ij", g("oooo"), t, t)
            X = np.einsum("ikce,cldj,klde->ij", t, g("vovo"), t)
            M += 0.5 * (X + X.T)
            M += 0.5 * np.einsum("cidj,klce,klde->ij", g("vovo"), t, t)
        return M

    def ip_m12(self):
        """Coupling block M[i, j, k, a] (1h row, 2h1p column) through order n-1."""
        g = self.blk
        M = np.einsum("jkia->ijka", g("ooov")).copy()
        if self.order >= 3:
            t = self.t2_1
            M -= 0.5 * np.einsum("aide,jkde->ijka", g("vovv"), t)
            X = np.einsum("ilkc,jlac->ijka", g("ooov"), t)
            M -= X - X.transpose(0, 2, 1, 3)
        return M

    def ip_m22(self):
        """2h1p-2h1p block M[i,j,a, k,l,b] through order n-2."""
        no, nv = self.no, self.nv
        I, J = np.eye(no), np.eye(nv)
        d = self.eo[:, None] + self.eo[None, :]
        M = np.einsum("ik,jl,ab->ijaklb", I, I, J) * (d[:, :, None, None, None, None] - self.ev[None, None, :, None, None, None])
        M = M - M.transpose(0, 1, 2, 4, 3, 5)
        if self.order >= 3:
            M = M - np.einsum("ab,ijkl->ijaklb", J, self.blk("oooo"))
            R = np.einsum("jl,kaib->ijaklb", I, self.blk("ovov"))
            R = R - R.transpose(1, 0, 2, 3, 4, 5)
            M = M + (R - R.transpose(0, 1, 2, 4, 3, 5))
        return M

    # ---- transition moments (Eqs. T_ea, T_ip, orders k + l <= torder) -------
    # First order vanishes in the one-particle columns.  Third order
    # (torder = 3, needs order >= 3) adds the cross terms of the second-order
    # density with t2(2), t1(3), the product t2(1) t1(2), and t2(2) in the
    # two-particle columns; the 2p1h (2h1p) columns get no other second-order
    # term.
    def ea_transition(self, torder=None):
        """T[p, nu] for p over all spin orbitals.

        Returns (T1 [nso, nv] for 1p columns, T2 [nso, o, v, v] for 2p1h columns).
        """
        torder = self.order if torder is None else torder
        t = self.t2_1
        no, nv = self.no, self.nv
        T1 = np.zeros((self.nso, nv))
        T1[no:] = np.eye(nv) - 0.25 * np.einsum("klcd,klbd->cb", t, t)
        T1[:no] = -self.t1_2
        T2 = np.zeros((self.nso, no, nv, nv))
        T2[:no] = t
        if torder >= 3:
            t2 = self.t2_2
            T1[no:] -= 0.25 * (np.einsum("klcd,klbd->cb", t, t2) + np.einsum("klcd,klbd->cb", t2, t))
            T1[:no] -= self.t1_3 + 0.5 * np.einsum("klbc,lc->kb", t, self.t1_2)
            T2[:no] += t2
        return T1, T2

    def ip_transition(self, torder=None):
        """T[p, nu]: (T1 [nso, o], T2 [nso, o, o, v])."""
        torder = self.order if torder is None else torder
        t = self.t2_1
        no, nv = self.no, self.nv
        T1 = np.zeros((self.nso, no))
        T1[:no] = np.eye(no) - 0.25 * np.einsum("klcd,jlcd->kj", t, t)
        T1[no:] = self.t1_2.T
        T2 = np.zeros((self.nso, no, no, nv))
        T2[no:] = t.transpose(2, 0, 1, 3)
        if torder >= 3:
            t2 = self.t2_2
            T1[:no] -= 0.25 * (np.einsum("klcd,jlcd->kj", t, t2) + np.einsum("klcd,jlcd->kj", t2, t))
            T1[no:] += self.t1_3.T + 0.5 * np.einsum("jlcd,ld->cj", t, self.t1_2)
            T2[no:] += t2.transpose(2, 0, 1, 3)
        return T1, T2

    # ---- dense matrix in the restricted basis ------------------------------
    def basis_labels(self, kind):
        no, nv = self.no, self.nv
        if kind == "ea":
            one = list(range(nv))
            two = [(i, a, b) for i in range(no) for a, b in combinations(range(nv), 2)]
        else:
            one = list(range(no))
            two = [(i, j, a) for a in range(nv) for i, j in combinations(range(no), 2)]
        return one, two

    def matrix(self, kind):
        """Dense ADC matrix in the restricted spin-orbital basis (fock.py ordering)."""
        one, two = self.basis_labels(kind)
        I = np.array(two)
        if kind == "ea":
            M11, M12, M22 = self.ea_m11(), self.ea_m12(), self.ea_m22()
            C = M12[:, I[:, 0], I[:, 1], I[:, 2]]
            D = M22[I[:, 0][:, None], I[:, 1][:, None], I[:, 2][:, None], I[:, 0][None, :], I[:, 1][None, :], I[:, 2][None, :]]
        else:
            M11, M12, M22 = self.ip_m11(), self.ip_m12(), self.ip_m22()
            C = M12[:, I[:, 0], I[:, 1], I[:, 2]]
            D = M22[I[:, 0][:, None], I[:, 1][:, None], I[:, 2][:, None], I[:, 0][None, :], I[:, 1][None, :], I[:, 2][None, :]]
        n1 = len(one)
        M = np.zeros((n1 + len(two), n1 + len(two)))
        M[:n1, :n1] = M11
        M[:n1, n1:] = C
        M[n1:, :n1] = C.T
        M[n1:, n1:] = D
        return M
