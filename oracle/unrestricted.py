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


def spin_orbital_df(sysm):
    """Spin-orbital DF factor B^Q_PR (block-diagonal in spin, order as above):
    (PR|QS) = sum_Q B^Q_PR B^Q_QS; returns (eps_so, no, B [naux, nso, nso])."""
    na, nb = sysm.nocc_a, sysm.nocc_b
    spin, idx = spin_orbital_order(sysm.nmo, na, nb)
    eps = np.where(spin == 0, np.asarray(sysm.eps_a)[idx], np.asarray(sysm.eps_b)[idx])
    B = np.stack([np.asarray(sysm.B_a, dtype=float), np.asarray(sysm.B_b, dtype=float)])
    Bso = B[spin[:, None], :, idx[:, None], idx[None, :]].transpose(2, 0, 1) * (spin[:, None] == spin[None, :])
    return eps, na + nb, Bso


class UnrestrictedDFADC:
    """Density-fitted EA/IP-UADC(n) of an unrestricted reference: the tier-1
    spin-orbital expressions with every integral that carries three or four
    virtual indices applied through B^Q (Eq. 19); nothing of size v^3 or v^4 is
    formed.  The o-containing blocks (ij|kl), (ij|ka), (ia|jb), (ij|ab) are
    formed from B^Q.  Notation as in tier 1 (spin orbitals, <pq||rs>); basis as
    in tier 1.  As in the spin-adapted oracle, IP applies M_IP = -M_- (lowest
    eigenvalues = lowest ionisation energies)."""

    def __init__(self, sysm, order=3, kind="ea"):
        assert order in (2, 3) and kind in ("ea", "ip")
        eps, no, B = spin_orbital_df(sysm)
        self.order = order
        self.kind = kind
        self.no = no
        self.nv = len(eps) - no
        o = slice(0, no)
        v = slice(no, len(eps))
        self.Boo, self.Bov, self.Bvv = B[:, o, o], B[:, o, v], B[:, v, v]
        self.eo, self.ev = eps[o], eps[v]
        e = lambda spec, *x: np.einsum(spec, *x, optimize=True)
        self.e = e
        self.ovov = e("Qia,Qjb->iajb", self.Bov, self.Bov)  # (ia|jb)
        self.oovv = e("Qij,Qab->ijab", self.Boo, self.Bvv)  # (ij|ab)
        self.oooo = e("Qij,Qkl->ijkl", self.Boo, self.Boo)  # (ij|kl)
        self.ooov = e("Qij,Qka->ijka", self.Boo, self.Bov)  # (ij|ka)
        self.D2 = self.eo[:, None, None, None] + self.eo[None, :, None, None] - self.ev[None, None, :, None] - self.ev[None, None, None, :]
        self.D1 = self.eo[:, None] - self.ev[None, :]
        self._amplitudes()
        # basis of tier 1: EA 1p a, 2p1h (i, a<b) i-major; IP 1h i, 2h1p (i<j, a) a-major
        from itertools import combinations

        if kind == "ea":
            self.n1 = self.nv
            two = [(i, a, b) for i in range(self.no) for a, b in combinations(range(self.nv), 2)]
            self.M11 = self.m11_ea()
        else:
            self.n1 = self.no
            two = [(i, j, a) for a in range(self.nv) for i, j in combinations(range(self.no), 2)]
            self.M11 = self.m11_ip()
            self.M12 = self.m12_ip()
        self.I = np.array(two, dtype=np.int64).reshape(-1, 3).T
        self.dim = self.n1 + self.I.shape[1]

    # <pq||rs> blocks with at most two virtual indices, from the chemists' blocks
    def g_oovv(self):  # <ij||ab> = (ia|jb) - (ib|ja)
        return np.einsum("iajb->ijab", self.ovov) - np.einsum("ibja->ijab", self.ovov)

    def g_oooo(self):  # <ij||kl> = (ik|jl) - (il|jk)
        return np.einsum("ikjl->ijkl", self.oooo) - np.einsum("iljk->ijkl", self.oooo)

    def g_ovvo(self):  # <ia||bj> = (ib|ja) - (ij|ab)
        return np.einsum("ibja->iabj", self.ovov) - np.einsum("ijab->iabj", self.oovv)

    def g_ooov(self):  # <ij||ka> = (ik|ja) - (ia|jk)
        return np.einsum("ikja->ijka", self.ooov) - np.einsum("jkia->ijka", self.ooov)

    def g_ovoo(self):  # <ia||jk> = (ij|ak) - (ik|aj)
        return np.einsum("ijka->iajk", self.ooov) - np.einsum("ikja->iajk", self.ooov)

    def ladder(self, X):
        """sum_cd (ac|bd) X[..., c, d] = sum_Q B^Q_vv X B^Q_vv (for X antisymmetric in cd this is
        1/2 sum_cd <ab||cd> X_cd)."""
        out = np.zeros_like(X)
        for BQ in self.Bvv:
            out += BQ @ X @ BQ
        return out

    def _amplitudes(self):
        e = self.e
        self.t2_1 = self.g_oovv() / self.D2
        t = self.t2_1
        if self.order < 3:
            self.t1_2 = self._singles(t) / self.D1
            return
        gov = self.g_ovvo()  # <kb||cj> = <kb||cj>
        X = e("kbcj,ikac->ijab", gov, t)
        ring = X - X.transpose(1, 0, 2, 3) - X.transpose(0, 1, 3, 2) + X.transpose(1, 0, 3, 2)
        num = self.ladder(t) + 0.5 * e("klij,klab->ijab", self.g_oooo(), t) + ring
        self.t2_2 = num / self.D2
        self.t1_2 = self._singles(t) / self.D1
        self.t1_3 = self._t1_third_order()

    def _singles(self, t):
        """-1/2 <ka||cd> t_ik^cd - 1/2 <kl||ic> t_kl^ac  (t antisymmetric)."""
        e = self.e
        # -1/2 <ka||cd> t_ik^cd = -sum <ka|cd> t_ik^cd = -sum (kc|ad) t_ik^cd
        s = -e("Qkc,Qad,ikcd->ia", self.Bov, self.Bvv, t)
        return s - 0.5 * e("klic,klac->ia", self.g_ooov(), t)

    def _t1_third_order(self):
        """t_i^a(3) of tier 1 (Eq. t_singles at k = 3) with every <vv||vo> through B^Q."""
        e, t, t1, t2 = self.e, self.t2_1, self.t1_2, self.t2_2
        Bov, Bvv = self.Bov, self.Bvv
        A = e("iajb,jb->ia", self.ovov, t1) - e("jiab,jb->ia", self.oovv, t1) + self._singles(t2)
        # <bc||dk> t_jk^bc = 2 (bd|ck) t_jk^bc
        Y = 2.0 * e("Qbd,Qkc,jkbc->jd", Bvv, Bov, t)
        E1 = e("ijad,jd->ia", t, Y)
        V = np.zeros((self.no, self.no, self.nv, self.no))
        for q in range(Bvv.shape[0]):
            W = np.tensordot(t, Bov[q], axes=([3], [1]))  # [j,k,b,i] = sum_c t_jk^bc B_ic
            V += np.tensordot(W, Bvv[q], axes=([2], [0])).transpose(0, 1, 3, 2)  # [j,k,d,i]
        E2 = 2.0 * e("jkad,jkdi->ia", t, V)
        R = e("ijbd,jkbc->ikcd", t, t)
        E3 = -(e("Qad,Qkc,ikcd->ia", Bvv, Bov, R) - e("Qka,Qcd,ikcd->ia", Bov, Bvv, R))
        rho = e("jkbc,jkbd->cd", t, t)
        E4 = -(e("Qad,Qic,cd->ia", Bvv, Bov, rho) - e("Qia,Qcd,cd->ia", Bov, Bvv, rho))
        gov = self.g_ovoo()
        F1 = e("ilab,jkbc,lcjk->ia", t, t, gov)
        F2 = -e("lcik,jkbc,jlab->ia", gov, t, t)
        F3 = e("lajk,jkbc,ilbc->ia", gov, t, t)
        F4 = -e("laik,jkbc,jlbc->ia", gov, t, t)
        W3 = 0.25 * (2 * E1 + E2 + 4 * E3 + 2 * E4) - 0.25 * (2 * F1 + 4 * F2 + F3 + 2 * F4)
        return (A + W3) / self.D1 + 0.5 * e("ijab,jb->ia", t, t1)

    def g_ovov(self):  # <ia||jb> = (ij|ab) - (ib|ja)
        return np.einsum("ijab->iajb", self.oovv) - np.einsum("ibja->iajb", self.ovov)

    def g_vovo(self):  # <ai||bj> = (ab|ij) - (aj|ib)
        return np.einsum("ijab->aibj", self.oovv) - np.einsum("jaib->aibj", self.ovov)

    def g_vooo(self):  # <ai||jk> = (aj|ik) - (ak|ij)
        return np.einsum("ikja->aijk", self.ooov) - np.einsum("ijka->aijk", self.ooov)

    # ---- one-particle blocks (tier-1 expressions, vvvv and ovvv through B^Q) ----
    def m11_ea(self):
        e, t = self.e, self.t2_1
        Bov, Bvv = self.Bov, self.Bvv
        M = np.diag(self.ev).copy()
        goovv = self.g_oovv()
        X = e("klac,klbc->ab", t, goovv)
        M -= 0.25 * (X + X.T)
        if self.order >= 3:
            t1, t2 = self.t1_2, self.t2_2
            # t_k^c <ka||cb>, <ka||cb> = (kc|ab) - (kb|ac)
            X = e("kc,Qkc,Qab->ab", t1, Bov, Bvv) - e("kc,Qkb,Qac->ab", t1, Bov, Bvv)
            M += X + X.T
            X = e("klac,klbc->ab", t2, goovv)
            M -= 0.25 * (X + X.T)
            # t_kl^ac <bc||de> t_kl^de = 2 t_kl^ac (ladder of t)_kl^bc
            X = 2.0 * e("klac,klbc->ab", t, self.ladder(t))
            M -= 0.125 * (X + X.T)
            # 1/2 <ac||bd> rho_cd, rho_cd = t_kl^ce t_kl^de, <ac||bd> = (ab|cd) - (ad|cb)
            rho = e("klce,klde->cd", t, t)
            M += 0.5 * (e("Qab,Qcd,cd->ab", Bvv, Bvv, rho) - e("Qad,Qcb,cd->ab", Bvv, Bvv, rho))
            gov = self.g_ovov()
            X = e("kmac,kdlb,lmcd->ab", t, gov, t)
            M -= 0.5 * (X + X.T)
            M -= 0.5 * e("kalb,kmcd,lmcd->ab", gov, t, t)
        return M

    def m11_ip(self):
        e, t = self.e, self.t2_1
        M = np.diag(self.eo).copy()
        goovv = self.g_oovv()
        X = e("ilcd,jlcd->ij", t, goovv)
        M += 0.25 * (X + X.T)
        if self.order >= 3:
            t1, t2 = self.t1_2, self.t2_2
            X = e("kc,cikj->ij", t1, self.g_vooo().transpose(0, 1, 2, 3))
            M += X + X.T
            X = e("ikcd,jkcd->ij", t2, goovv)
            M += 0.25 * (X + X.T)
            goooo = self.g_oooo()
            X = e("ikcd,jklm,lmcd->ij", t, goooo, t)
            M += 0.125 * (X + X.T)
            M -= 0.5 * e("ikjl,kmcd,lmcd->ij", goooo, t, t)
            gvovo = self.g_vovo()
            X = e("ikce,cldj,klde->ij", t, gvovo, t)
            M += 0.5 * (X + X.T)
            M += 0.5 * e("cidj,klce,klde->ij", gvovo, t, t)
        return M

    def m12_ip(self):
        """Coupling M[i, j, k, a] (1h row, 2h1p column) through order n-1, explicit (o^3 v)."""
        e, t = self.e, self.t2_1
        M = np.einsum("jkia->ijka", self.g_ooov()).copy()
        if self.order >= 3:
            # 1/2 <ai||de> t_jk^de = (ad|ie) t_jk^de: sum_e B^Q_ie t_jk^de, then sum_Qd B^Q_ad
            G = np.tensordot(self.Bov, t, axes=([2], [3]))  # [Q,i,j,k,d]
            M -= np.tensordot(G, self.Bvv, axes=([0, 4], [0, 2]))  # [i,j,k,a]
            X = e("ilkc,jlac->ijka", self.g_ooov(), t)
            M -= X - X.transpose(0, 2, 1, 3)
        return M

    # ---- sigma = M Y (two-particle block and EA coupling applied, not formed) ----
    def _full(self, y2):
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
        e = self.e
        y1, F = Y[:, : self.n1], self._full(Y[:, self.n1 :])
        s1 = y1 @ self.M11.T
        if self.kind == "ea":
            Bov, Bvv, t = self.Bov, self.Bvv, self.t2_1
            # coupling, first order: M12[a,j,c,d] = -<aj||cd> = -[(ac|jd) - (ad|jc)]
            s1 -= e("Qac,Qjd,njcd->na", Bvv, Bov, F)
            P = e("na,Qac->nQc", y1, Bvv)
            S2 = -(e("nQc,Qjd->njcd", P, Bov) - e("nQd,Qjc->njcd", P, Bov))
            if self.order >= 3:
                gvooo = self.g_vooo()
                # -1/2 <aj||lm> t_lm^cd
                G = e("lmcd,njcd->njlm", t, F)
                s1 -= 0.25 * e("ajlm,njlm->na", gvooo, G)
                U = e("na,ajlm->njlm", y1, gvooo)
                S2 -= 0.5 * e("njlm,lmcd->njcd", U, t)
                # -(X - X^cd), X[a,j,c,d] = <ae||cm> t_jm^de, <ae||cm> = (ac|em) - (am|ec)
                H = e("jmde,njcd->nmec", t, F)
                s1 -= e("Qac,Qme,nmec->na", Bvv, Bov, H) - e("Qma,Qec,nmec->na", Bov, Bvv, H)
                K = e("nQc,Qme->necm", P, Bov) - e("na,Qma,Qec->necm", y1, Bov, Bvv)
                X = e("necm,jmde->njcd", K, t)
                S2 -= X - X.transpose(0, 1, 3, 2)
            S2 += (self.ev[None, None, :, None] + self.ev[None, None, None, :] - self.eo[None, :, None, None]) * F
            if self.order >= 3:
                for BQ in Bvv:
                    S2 += BQ @ F @ BQ
                R = e("ajci,njcb->niab", self.g_vovo(), F)
                S2 -= R - R.transpose(0, 1, 3, 2)
        else:
            s1 += 0.5 * e("ijka,njka->ni", self.M12, F)
            S2 = e("ijka,ni->njka", self.M12, y1)
            S2 += (self.eo[None, :, None, None] + self.eo[None, None, :, None] - self.ev[None, None, None, :]) * F
            if self.order >= 3:
                S2 -= 0.5 * e("ijkl,nkla->nija", self.g_oooo(), F)
                R = e("kaib,nkjb->nija", self.g_ovov(), F)
                S2 += R - R.transpose(0, 2, 1, 3)
        i0, i1, i2 = self.I
        out = np.concatenate([s1, S2[:, i0, i1, i2]], axis=1)
        return out if self.kind == "ea" else -out

    def dense(self):
        return self.sigma(np.eye(self.dim)).T

    def spectroscopic_factors(self, Y, torder=None):
        """P_mu = sum_p |X_p mu|^2 (Eq. spec_factors, one spin-orbital component,
        so a Koopmans state has P = 1) for rows of Y normalised here, with T
        through order torder (default n) from the tier-1 expressions
        (Eqs. T_ea, T_ip), which need only the amplitudes."""
        from oracle.spinorb import SpinOrbitalADC

        Y = np.atleast_2d(np.asarray(Y, dtype=float))
        Y = Y / np.linalg.norm(Y, axis=1)[:, None]
        self.nso = self.no + self.nv
        tr = SpinOrbitalADC.ea_transition if self.kind == "ea" else SpinOrbitalADC.ip_transition
        T1, T2 = tr(self, torder)
        i0, i1, i2 = self.I
        T = np.concatenate([T1, T2[:, i0, i1, i2]], axis=1)
        X = Y @ T.T
        return np.einsum("rp,rp->r", X, X)

    def apply_S(self, Y):
        return np.array(Y, dtype=float)

    def solve_S(self, Y):
        return np.array(Y, dtype=float)

    def diagonal(self):
        i0, i1, i2 = self.I
        if self.kind == "ea":
            return np.concatenate([np.diag(self.M11), self.ev[i1] + self.ev[i2] - self.eo[i0]])
        return -np.concatenate([np.diag(self.M11), self.eo[i0] + self.eo[i1] - self.ev[i2]])
