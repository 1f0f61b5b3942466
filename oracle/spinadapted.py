"""Tier-2 oracle: spin-adapted, density-fitted EA/IP-ADC(n) (n = 2, 3), matrix-free.
TEST INFRASTRUCTURE ONLY -- nothing in the GPU product path may import this.

Spin adaptation (Sec. III B).  Closed-shell doublet vectors:
  EA  Y = [Y_a (v) | Y_iab (o*v*v, b fastest)]
  IP  Y = [Y_i (o) | Y_ija (o*o*v, a fastest)]
Y_iab is the amplitude of the mixed-spin 2p1h determinant (i_b, a_b, b_a) and
Y_iab - Y_iba that of the all-alpha one (the EA mirror of Eqs. M_ijka1/2,
M_ilbjka1/2, T_jka1/2); likewise Y_ija <-> (i_b j_a a_b) for IP.  With this
embedding E the metric is S = E^T E = diag(1, 2 - P) (P swaps the two like
indices), which reproduces the norm of the Appendix (Eq. appendix_3), and the
spin-adapted product is sigma = S^-1 E^T M E Y; its 1p/1h row has the
(2 Y - P Y) weighting of Eq. sigma_i_adapted_3 and its 2p1h/2h1p row is the
mixed-spin component (Eq. sigma_jka_bab).

Density fitting (Sec. III C, Eq. 19): (pq|rs) = sum_Q B^Q_pq B^Q_rs.  The
vvvv (EA) block is never formed: its terms are evaluated as
sum_Q B^Q X B^Q.  All other integrals are formed from B when needed.

Sign convention for IP: the matrix applied here is M_IP = -M_- (the negative
of the paper's Eq. M_ip matrix), so that its lowest eigenvalues are the lowest
ionisation energies E_{N-1} - E_N.  EA uses M_+ itself (eigenvalues
E_{N+1} - E_N; the paper's electron affinity is the negative, Sec. IV).

The spatial working equations below were obtained by integrating the spin-
orbital equations of ``spinorb.py`` over spin (Eqs. eps_spin_adapted ...
t_aaaa) and are checked term by term against them through the embedding.
Notation: (pq|rs) chemists' integrals, t_ij^ab = t[i,j,a,b] (alpha-beta
component), D_ij^ab = e_i + e_j - e_a - e_b, D_i^a = e_i - e_a.
"""
from __future__ import annotations

import numpy as np


def df_ladder(Bvv, X):
    """sum_cd (ac|bd) X[..., c, d] with (ac|bd) = sum_Q B^Q_ac B^Q_bd (Eq. 19): sum_Q B^Q X B^Q.

    Written as a loop over the auxiliary index so that no intermediate larger
    than X is formed."""
    X = np.asarray(X, dtype=np.float64)
    out = np.zeros_like(X)
    for BQ in Bvv:
        out += BQ @ X @ BQ
    return out


class SpinAdaptedADC:
    """Closed-shell DF-ADC(order) for EA (kind='ea') or IP (kind='ip')."""

    def __init__(self, eps, nocc, B, order=3, kind="ea"):
        assert order in (2, 3) and kind in ("ea", "ip")
        self.eps = np.asarray(eps, dtype=np.float64)
        self.o = nocc
        self.v = len(self.eps) - nocc
        self.order = order
        self.kind = kind
        B = np.asarray(B, dtype=np.float64)
        o = nocc
        self.Boo = np.ascontiguousarray(B[:, :o, :o])
        self.Bov = np.ascontiguousarray(B[:, :o, o:])
        self.Bvv = np.ascontiguousarray(B[:, o:, o:])
        self.eo = self.eps[:o]
        self.ev = self.eps[o:]
        self._integrals()
        self._amplitudes()
        self.M11 = self._m11()

    # ---- integrals from the DF factors (Eq. 19) ---------------------------
    def _integrals(self):
        Boo, Bov, Bvv = self.Boo, self.Bov, self.Bvv
        self.ovov = np.einsum("Qia,Qjb->iajb", Bov, Bov, optimize=True)  # (ia|jb)
        self.oovv = np.einsum("Qij,Qab->ijab", Boo, Bvv, optimize=True)  # (ij|ab)
        self.oooo = np.einsum("Qij,Qkl->ijkl", Boo, Boo, optimize=True)  # (ij|kl)
        self.ooov = np.einsum("Qij,Qka->ijka", Boo, Bov, optimize=True)  # (ij|ka)

    def ladder(self, X):
        """sum_cd (ac|bd) X[..., c, d] = sum_Q (B^Q X B^Q)_ab  (vvvv never stored)."""
        return df_ladder(self.Bvv, X)

    def ovvv_contract(self, X, pattern):
        """Contractions with the (ov|vv) class through B, never forming it."""
        return np.einsum(pattern, self.Bov, self.Bvv, X, optimize=True)

    # ---- amplitudes (Eqs. t_singles, t_doubles; MP-equivalent) ------------
    def _amplitudes(self):
        eo, ev = self.eo, self.ev
        D2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
        D1 = eo[:, None] - ev[None, :]
        self.D2, self.D1 = D2, D1
        ovov, oovv, oooo = self.ovov, self.oovv, self.oooo
        t = ovov.transpose(0, 2, 1, 3) / D2  # t_ij^ab = (ia|jb)/D
        self.t = t
        if self.order < 3:
            return
        # second-order doubles: D t = sum_cd (ac|bd) t_ij^cd + sum_kl (ki|lj) t_kl^ab + W + W^T
        lad = self.ladder(t)
        hh = np.einsum("kilj,klab->ijab", oooo, t, optimize=True)
        W = (
            2.0 * np.einsum("kcjb,ikac->ijab", ovov, t, optimize=True)
            - np.einsum("kcjb,ikca->ijab", ovov, t, optimize=True)
            - np.einsum("kjbc,ikac->ijab", oovv, t, optimize=True)
            - np.einsum("kjac,ikcb->ijab", oovv, t, optimize=True)
        )
        self.t_2 = (lad + hh + W + W.transpose(1, 0, 3, 2)) / D2
        # second-order singles: D t_i^a = sum (kc|ad)(2 t_ik^dc - t_ik^cd) - sum (ki|lc)(2 t_kl^ac - t_kl^ca)
        tau = 2.0 * t - t.transpose(0, 1, 3, 2)
        s1 = self.ovvv_contract(tau, "Qkc,Qad,ikdc->ia")
        s2 = np.einsum("kilc,klac->ia", self.ooov, tau, optimize=True)
        self.t1_2 = (s1 - s2) / D1
        self.t1_3 = self._t1_third_order()

    def _t1_third_order(self):
        """Third-order singles t_i^a(3) (Eq. t_singles at k = 3), spin-integrated.

        Spin-orbital form: D t(3) = A + 1/4 t_jk^bc W_ijk^abc, plus
        1/2 t_ij^ab t_j^b(2) after the division (A: the t1(2) and t2(2) singles
        terms; W: connected first-order triples).  Integrating over spin with
        tau = 2t - t(ab swapped), u = t - t(ab swapped) gives, term for term,
          A1 = sum [2 (ia|jb) - (ij|ab)] t_j^b(2)
          A2 = the t1(2) expression with tau(2) built from t2(2)
          E1 = sum tau_ij^ad Y_jd,  Y_jd = 2 sum tau_jk^bc (bd|kc)
          E2 = -4 sum t_jk^ad tau_jk^cb (bd|ic)
          E3 = sum (ad|kc) R1_ik^dc + sum (ka|cd) R2_ik^cd
          E4 = sum rho_cd [2 (ia|cd) - (ad|ic)],  rho_cd = 2 sum t_jk^cb tau_jk^db
          F1 = sum tau_il^ab Z_lb,  Z_lb = 2 sum tau_jk^bc (lj|kc)
          F2 = sum (li|kc) R1_lk^ac + sum (lk|ic) R2_lk^ca
          F3 = 4 sum (lj|ka) X_jkil,  X_jkil = sum t_jk^bc u_il^bc - t_kj^bc t_il^bc
          F4 = sum rho'_kl [2 (lk|ia) - (li|ka)],  rho'_kl = 2 sum t_jk^bc tau_jl^bc
        with the ring products R1_ik^dc = sum tau_ij^db tau_jk^bc and
        R2_ik^cd = -sum (tau_ij^db t_jk^bc + tau_ij^bd t_jk^cb), and
        D t(3) = A1 + A2 + (2 E1 + E2 + 4 E3 + 2 E4)/4 - (2 F1 + 4 F2 + F3 + 2 F4)/4.
        """
        t, t1, t2 = self.t, self.t1_2, self.t_2
        Boo, Bov, Bvv = self.Boo, self.Bov, self.Bvv

        def e(spec, *ops):
            return np.einsum(spec, *ops, optimize=True)

        sw = (0, 1, 3, 2)
        tau = 2.0 * t - t.transpose(sw)
        u = t - t.transpose(sw)
        tau2 = 2.0 * t2 - t2.transpose(sw)
        A1 = 2.0 * e("iajb,jb->ia", self.ovov, t1) - e("jiab,jb->ia", self.oovv, t1)
        A2 = self.ovvv_contract(tau2, "Qkc,Qad,ikdc->ia") - e("kilc,klac->ia", self.ooov, tau2)
        E1 = e("ijad,jd->ia", tau, 2.0 * self.ovvv_contract(tau, "Qkc,Qbd,jkbc->jd"))
        # E2 one auxiliary index at a time: V_jkdi = sum_Q sum_b B^Q_db sum_c tau_jk^cb B^Q_ic
        V = np.zeros((self.o, self.o, self.v, self.o))
        for q in range(Boo.shape[0]):
            Wq = np.tensordot(tau, Bov[q], axes=([2], [1]))  # [j,k,b,i]
            V += np.tensordot(Wq, Bvv[q], axes=([2], [1])).transpose(0, 1, 3, 2)  # [j,k,d,i]
        E2 = -4.0 * e("jkad,jkdi->ia", t, V)
        R1 = e("ijdb,jkbc->ikdc", tau, tau)
        R2 = -e("ijdb,jkbc->ikcd", tau, t) - e("ijbd,jkcb->ikcd", tau, t)
        E3 = e("Qad,Qkc,ikdc->ia", Bvv, Bov, R1) + e("Qka,Qcd,ikcd->ia", Bov, Bvv, R2)
        rho = 2.0 * e("jkcb,jkdb->cd", t, tau)
        E4 = 2.0 * e("Qia,Qcd,cd->ia", Bov, Bvv, rho) - e("Qad,Qic,cd->ia", Bvv, Bov, rho)
        F1 = e("ilab,lb->ia", tau, 2.0 * e("Qlj,Qkc,jkbc->lb", Boo, Bov, tau))
        F2 = e("Qli,Qkc,lkac->ia", Boo, Bov, R1) + e("Qlk,Qic,lkca->ia", Boo, Bov, R2)
        X = e("jkbc,ilbc->jkil", t, u) - e("kjbc,ilbc->jkil", t, t)
        F3 = 4.0 * e("ljka,jkil->ia", self.ooov, X)
        rhoh = 2.0 * e("jkbc,jlbc->kl", t, tau)
        F4 = 2.0 * e("lkia,kl->ia", self.ooov, rhoh) - e("lika,kl->ia", self.ooov, rhoh)
        num = A1 + A2 + 0.25 * (2.0 * E1 + E2 + 4.0 * E3 + 2.0 * E4) - 0.25 * (2.0 * F1 + 4.0 * F2 + F3 + 2.0 * F4)
        return num / self.D1 + 0.5 * e("ijab,jb->ia", tau, t1)

    def mp_energies(self):
        """MP correlation energy through order n (Sec. III A step 2), spin-integrated:
        E(2) = sum (ia|jb)(2 t_ij^ab - t_ij^ba), E(3) the same with t2(2)."""
        out = []
        for t in (self.t, getattr(self, "t_2", None))[: self.order - 1]:
            out.append(float(np.einsum("iajb,ijab->", self.ovov, 2.0 * t - t.transpose(0, 1, 3, 2))))
        return out

    # ---- 1p-1p / 1h-1h block (Table 1 second row; precomputed, Sec. III A) --
    def _m11(self):
        return self._m11_ea() if self.kind == "ea" else -self._m11_ip()

    def _m11_ea(self):
        t = self.t
        ovov = self.ovov
        M = np.diag(self.ev).copy()

        def sym(X):
            return X + X.T

        # second order: -sum t_kl^ac [(kb|lc) - 1/2 (kc|lb)] + (a<->b)
        M += sym(-np.einsum("klac,kblc->ab", t, ovov, optimize=True) + 0.5 * np.einsum("klac,kclb->ab", t, ovov, optimize=True))
        if self.order < 3:
            return M
        t2, t1 = self.t_2, self.t1_2
        Bov, Bvv = self.Bov, self.Bvv
        # t1(2) terms: sum_kc t_k^c [2 (kc|ab) - (kb|ac)] + (a<->b)
        K1 = 2.0 * np.einsum("Qkc,kc,Qab->ab", Bov, t1, Bvv, optimize=True) - np.einsum("Qkb,kc,Qac->ab", Bov, t1, Bvv, optimize=True)
        M += sym(K1)
        # t2(2) terms, same shape as second order
        M += sym(-np.einsum("klac,kblc->ab", t2, ovov, optimize=True) + 0.5 * np.einsum("klac,kclb->ab", t2, ovov, optimize=True))
        # vvvv with one open line: -sum t_kl^ac [L_kl^bc - 1/2 L_kl^cb], L_kl = sum_Q B^Q t_kl B^Q
        L = self.ladder(t)
        M += sym(-np.einsum("klac,klbc->ab", t, L, optimize=True) + 0.5 * np.einsum("klac,klcb->ab", t, L, optimize=True))
        # vvvv with both lines on the integral: sum_cd [2 (ab|cd) - (ad|cb)] (2X - X')_cd
        X = np.einsum("klce,klde->cd", t, t, optimize=True)
        Xp = np.einsum("klce,kled->cd", t, t, optimize=True)
        Z = 2.0 * X - Xp
        M += 2.0 * np.einsum("Qab,Qcd,cd->ab", Bvv, Bvv, Z, optimize=True) - np.einsum("Qad,cd,Qcb->ab", Bvv, Z, Bvv, optimize=True)
        # ring with one open line on each amplitude / on the integral
        oovv = self.oovv  # (kl|db) -> oovv[k,l,d,b]
        Y5 = (
            -0.5 * np.einsum("kmac,kldb,lmcd->ab", t, oovv, t, optimize=True)
            + 1.0 * np.einsum("kmac,kldb,lmdc->ab", t, oovv, t, optimize=True)
            + 1.0 * np.einsum("kmac,kbld,lmcd->ab", t, ovov, t, optimize=True)
            - 2.0 * np.einsum("kmac,kbld,lmdc->ab", t, ovov, t, optimize=True)
            + 1.0 * np.einsum("kmca,kldb,lmcd->ab", t, oovv, t, optimize=True)
            - 0.5 * np.einsum("kmca,kldb,lmdc->ab", t, oovv, t, optimize=True)
            - 0.5 * np.einsum("kmca,kbld,lmcd->ab", t, ovov, t, optimize=True)
            + 1.0 * np.einsum("kmca,kbld,lmdc->ab", t, ovov, t, optimize=True)
        )
        M += sym(Y5)
        # ring with both lines on the integral: -sum_kl [2 (kl|ab) - (kb|la)] (2U - U')_kl
        U = np.einsum("kmcd,lmcd->kl", t, t, optimize=True)
        Up = np.einsum("kmcd,lmdc->kl", t, t, optimize=True)
        V = 2.0 * U - Up
        M -= 2.0 * np.einsum("klab,kl->ab", oovv, V, optimize=True) - np.einsum("kbla,kl->ab", ovov, V, optimize=True)
        return M

    def _m11_ip(self):
        """Paper's M_- 1h-1h block (the class applies the overall sign)."""
        t = self.t
        ovov = self.ovov
        M = np.diag(self.eo).copy()

        def sym(X):
            return X + X.T

        # second order: sum t_il^cd [(jc|ld) - 1/2 (jd|lc)] + (i<->j)
        M += sym(np.einsum("ilcd,jcld->ij", t, ovov, optimize=True) - 0.5 * np.einsum("ilcd,jdlc->ij", t, ovov, optimize=True))
        if self.order < 3:
            return M
        t2, t1 = self.t_2, self.t1_2
        oooo, oovv, ooov = self.oooo, self.oovv, self.ooov
        # t1(2): sum_kc t_k^c [2 (ck|ij) - (cj|ik)] + (i<->j)
        K1 = 2.0 * np.einsum("kc,ijkc->ij", t1, ooov, optimize=True) - np.einsum("kc,ikjc->ij", t1, ooov, optimize=True)
        M += sym(K1)
        # t2(2): sum t2_ik^cd [(cj|dk) - 1/2 (ck|dj)] + (i<->j)
        M += sym(np.einsum("ikcd,jckd->ij", t2, ovov, optimize=True) - 0.5 * np.einsum("ikcd,kcjd->ij", t2, ovov, optimize=True))
        # oooo with one open line: sum t_ik^cd (jl|km) [t_lm^cd - 1/2 t_lm^dc] + (i<->j)
        tau_h = t - 0.5 * t.transpose(0, 1, 3, 2)
        M += sym(np.einsum("ikcd,jlkm,lmcd->ij", t, oooo, tau_h, optimize=True))
        # oooo both lines on the integral: -[2 (ij|kl) - (il|kj)] (2U - U')_kl
        U = np.einsum("kmcd,lmcd->kl", t, t, optimize=True)
        Up = np.einsum("kmcd,lmdc->kl", t, t, optimize=True)
        V = 2.0 * U - Up
        M -= 2.0 * np.einsum("ijkl,kl->ij", oooo, V, optimize=True) - np.einsum("ilkj,kl->ij", oooo, V, optimize=True)
        # ring with open lines on the amplitudes: integrals (cd|lj) = oovv[l,j,c,d], (cj|ld) = ovov[j,c,l,d]
        Y5 = (
            0.5 * np.einsum("ikce,ljcd,klde->ij", t, oovv, t, optimize=True)
            - 1.0 * np.einsum("ikce,ljcd,kled->ij", t, oovv, t, optimize=True)
            - 1.0 * np.einsum("ikce,jcld,klde->ij", t, ovov, t, optimize=True)
            + 2.0 * np.einsum("ikce,jcld,kled->ij", t, ovov, t, optimize=True)
            - 1.0 * np.einsum("ikec,ljcd,klde->ij", t, oovv, t, optimize=True)
            + 0.5 * np.einsum("ikec,ljcd,kled->ij", t, oovv, t, optimize=True)
            + 0.5 * np.einsum("ikec,jcld,klde->ij", t, ovov, t, optimize=True)
            - 1.0 * np.einsum("ikec,jcld,kled->ij", t, ovov, t, optimize=True)
        )
        M += sym(Y5)
        # ring both lines on the integral: [2 (cd|ij) - (cj|id)] (2X - X')_cd
        X = np.einsum("klce,klde->cd", t, t, optimize=True)
        Xp = np.einsum("klce,kled->cd", t, t, optimize=True)
        Z = 2.0 * X - Xp
        M += 2.0 * np.einsum("ijcd,cd->ij", oovv, Z, optimize=True) - np.einsum("jcid,cd->ij", ovov, Z, optimize=True)
        return M

    # ---- dimensions, metric, diagonal -------------------------------------
    @property
    def n1(self):
        return self.v if self.kind == "ea" else self.o

    @property
    def dim(self):
        o, v = self.o, self.v
        return v + o * v * v if self.kind == "ea" else o + o * o * v

    def _split(self, Y):
        o, v = self.o, self.v
        Y = np.asarray(Y, dtype=np.float64)
        n1 = self.n1
        shp = (o, v, v) if self.kind == "ea" else (o, o, v)
        return Y[..., :n1], Y[..., n1:].reshape(Y.shape[:-1] + shp)

    def _swap(self, Y2):
        """The permutation P of the metric: swaps the two like indices."""
        return np.swapaxes(Y2, -1, -2) if self.kind == "ea" else np.swapaxes(Y2, -3, -2)

    def apply_S(self, Y):
        """S Y with S = E^T E = diag(1, 2 - P) (Appendix norm, Eq. appendix_3)."""
        y1, y2 = self._split(Y)
        return np.concatenate([y1, (2.0 * y2 - self._swap(y2)).reshape(y1.shape[:-1] + (-1,))], axis=-1)

    def solve_S(self, Y):
        """S^-1 Y: on each like-index pair (2 - P)^-1 = (2 + P)/3."""
        y1, y2 = self._split(Y)
        return np.concatenate([y1, ((2.0 * y2 + self._swap(y2)) / 3.0).reshape(y1.shape[:-1] + (-1,))], axis=-1)

    def diagonal(self):
        """Zeroth-order diagonal of the 2p1h/2h1p block and diag(M_11)."""
        o, v = self.o, self.v
        if self.kind == "ea":
            d2 = self.ev[None, :, None] + self.ev[None, None, :] - self.eo[:, None, None]
        else:
            d2 = self.ev[None, None, :] - self.eo[:, None, None] - self.eo[None, :, None]
        return np.concatenate([np.diag(self.M11), d2.ravel()])

    # ---- the sigma vector (Eqs. sigma_i_adapted_3, sigma_jka_bab) ----------
    def coupling_row(self, Y2):
        """1p (1h) row applied to the 2p1h (2h1p) part: sum M_{p,...} (2Y - PY)."""
        Yt = 2.0 * Y2 - self._swap(Y2)
        return self._cpl_ea_row(Yt) if self.kind == "ea" else -self._cpl_ip_row(Yt)

    def coupling_col(self, y1):
        """2p1h (2h1p) rows applied to the 1p (1h) part: sum_p M_{p,...} Y_p."""
        return self._cpl_ea_col(y1) if self.kind == "ea" else -self._cpl_ip_col(y1)

    def block22(self, Y2):
        return self._m22_ea(Y2) if self.kind == "ea" else -self._m22_ip(Y2)

    def sigma(self, Y):
        """sigma = M Y for Y of shape [dim] or [nvec, dim]."""
        y1, y2 = self._split(Y)
        s1 = y1 @ self.M11.T + self.coupling_row(y2)
        s2 = self.coupling_col(y1) + self.block22(y2)
        return np.concatenate([s1, s2.reshape(y1.shape[:-1] + (-1,))], axis=-1)

    # EA coupling tensor M_{a,jcd} =
    #   (ad|jc)                                          [first order]
    # + sum_lm (al|jm) t_lm^dc + sum_me (ad|em)(2 t_jm^ce - t_jm^ec)
    # - sum_me (am|ed) t_jm^ce - sum_me (am|ec) t_jm^ed    [second order]
    def _cpl_ea_row(self, Yt):
        Bov, Bvv, Boo = self.Bov, self.Bvv, self.Boo
        s = np.einsum("Qad,Qjc,...jcd->...a", Bvv, Bov, Yt, optimize=True)
        if self.order >= 3:
            t = self.t
            tau = 2.0 * t - t.transpose(0, 1, 3, 2)
            Z = np.einsum("lmdc,...jcd->...lmj", t, Yt, optimize=True)
            s = s + np.einsum("Qla,Qjm,...lmj->...a", Bov, Boo, Z, optimize=True)
            V = np.einsum("jmce,...jcd->...med", tau, Yt, optimize=True)
            s = s + np.einsum("Qad,Qme,...med->...a", Bvv, Bov, V, optimize=True)
            U = np.einsum("jmce,...jcd->...med", t, Yt, optimize=True)
            s = s - np.einsum("Qma,Qed,...med->...a", Bov, Bvv, U, optimize=True)
            U2 = np.einsum("jmed,...jcd->...mec", t, Yt, optimize=True)
            s = s - np.einsum("Qma,Qec,...mec->...a", Bov, Bvv, U2, optimize=True)
        return s

    def _cpl_ea_col(self, y1):
        Bov, Bvv, Boo = self.Bov, self.Bvv, self.Boo
        # sigma_iab += sum_c M_{c,iab} Y_c
        s = np.einsum("Qcb,Qia,...c->...iab", Bvv, Bov, y1, optimize=True)
        if self.order >= 3:
            t = self.t
            tau = 2.0 * t - t.transpose(0, 1, 3, 2)
            P = np.einsum("Qlc,Qim,...c->...lim", Bov, Boo, y1, optimize=True)  # sum_c (cl|im) Y_c
            s = s + np.einsum("...lim,lmba->...iab", P, t, optimize=True)
            q = np.einsum("Qcb,Qme,...c->...bme", Bvv, Bov, y1, optimize=True)  # sum_c (cb|em) Y_c
            s = s + np.einsum("...bme,imae->...iab", q, tau, optimize=True)
            r = np.einsum("Qmc,Qeb,...c->...meb", Bov, Bvv, y1, optimize=True)  # sum_c (cm|eb) Y_c
            s = s - np.einsum("...meb,imae->...iab", r, t, optimize=True)
            s = s - np.einsum("...mea,imeb->...iab", r, t, optimize=True)
        return s

    def _m22_ea(self, Y2):
        o, v = self.o, self.v
        d = self.ev[None, :, None] + self.ev[None, None, :] - self.eo[:, None, None]
        s = d * Y2
        if self.order >= 3:
            s = s + self.ladder(Y2)  # sum_cd (ac|bd) Y_icd
            oovv, ovov = self.oovv, self.ovov
            s = s - np.einsum("jiac,...jcb->...iab", oovv, Y2, optimize=True)  # (ac|ji) Y_jcb
            s = s + 2.0 * np.einsum("iajc,...jcb->...iab", ovov, Y2, optimize=True)  # (ai|jc) Y_jcb
            s = s - np.einsum("iajc,...jbc->...iab", ovov, Y2, optimize=True)  # (ai|jc) Y_jbc
            s = s - np.einsum("jibd,...jad->...iab", oovv, Y2, optimize=True)  # (bd|ji) Y_jad
        return s

    # IP coupling tensor (paper's M_-) M_{i,jka} =
    #   -(ki|ja)                                                      [first order]
    # - sum_de (ad|ie) t_jk^de - sum_lc (ik|lc)(2 t_jl^ac - t_jl^ca)
    # + sum_lc (ic|lk) t_jl^ac + sum_lc (ic|lj) t_kl^ca                [second order]
    def _cpl_ip_row(self, Yt):
        Bov, Boo = self.Bov, self.Boo
        s = -np.einsum("Qki,Qja,...jka->...i", Boo, Bov, Yt, optimize=True)
        if self.order >= 3:
            t = self.t
            tau = 2.0 * t - t.transpose(0, 1, 3, 2)
            Z = np.einsum("jkde,...jka->...dea", t, Yt, optimize=True)
            s = s - np.einsum("Qie,Qad,...dea->...i", Bov, self.Bvv, Z, optimize=True)
            ooov = self.ooov  # (ik|lc) = ooov[i,k,l,c]
            s = s - np.einsum("iklc,jlac,...jka->...i", ooov, tau, Yt, optimize=True)
            s = s + np.einsum("lkic,jlac,...jka->...i", ooov, t, Yt, optimize=True)
            s = s + np.einsum("ljic,klca,...jka->...i", ooov, t, Yt, optimize=True)
        return s

    def _cpl_ip_col(self, y1):
        Bov, Boo = self.Bov, self.Boo
        s = -np.einsum("Qki,Qja,...i->...jka", Boo, Bov, y1, optimize=True)
        if self.order >= 3:
            t = self.t
            tau = 2.0 * t - t.transpose(0, 1, 3, 2)
            w = np.einsum("Qie,Qad,...i->...ead", Bov, self.Bvv, y1, optimize=True)  # sum_i (ad|ie) Y_i
            s = s - np.einsum("...ead,jkde->...jka", w, t, optimize=True)
            ooov = self.ooov
            s = s - np.einsum("iklc,jlac,...i->...jka", ooov, tau, y1, optimize=True)
            s = s + np.einsum("lkic,jlac,...i->...jka", ooov, t, y1, optimize=True)
            s = s + np.einsum("ljic,klca,...i->...jka", ooov, t, y1, optimize=True)
        return s

    def _m22_ip(self, Y2):
        d = self.eo[:, None, None] + self.eo[None, :, None] - self.ev[None, None, :]
        s = d * Y2
        if self.order >= 3:
            oooo, oovv, ovov = self.oooo, self.oovv, self.ovov
            s = s - np.einsum("kilj,...kla->...ija", oooo, Y2, optimize=True)
            s = s + np.einsum("kiab,...kjb->...ija", oovv, Y2, optimize=True)
            s = s - 2.0 * np.einsum("iakb,...kjb->...ija", ovov, Y2, optimize=True)
            s = s + np.einsum("iakb,...jkb->...ija", ovov, Y2, optimize=True)
            s = s + np.einsum("kjab,...ikb->...ija", oovv, Y2, optimize=True)
        return s

    # ---- dense matrix (small systems only) ---------------------------------
    def dense(self):
        """M as a dense [dim, dim] array (columns sigma(e_k))."""
        I = np.eye(self.dim)
        return self.sigma(I).T


def embedding(nocc, nvir, kind):
    """E: spin-adapted vector -> spin-orbital vector in the restricted basis of
    ``spinorb.SpinOrbitalADC.basis_labels`` (spin orbital P = 2p + s, s=1 beta).

    EA: Y_a -> (a_alpha); Y_iab -> mixed (i_b, a_b, b_a) with weight 1 and the
    all-alpha (i_a, a_a, b_a) with Y_iab - Y_iba.  IP: Y_i -> (i_alpha);
    Y_jka -> (j_b, k_a, a_b) and all-alpha Y_jka - Y_kja.
    """
    from itertools import combinations

    o, v = nocc, nvir
    NO, NV = 2 * o, 2 * v
    if kind == "ea":
        two = [(i, a, b) for i in range(NO) for a, b in combinations(range(NV), 2)]
        n1, nso1 = v, NV
    else:
        two = [(i, j, a) for a in range(NV) for i, j in combinations(range(NO), 2)]
        n1, nso1 = o, NO
    pos = {lab: k for k, lab in enumerate(two)}
    dim = n1 + (o * v * v if kind == "ea" else o * o * v)
    E = np.zeros((nso1 + len(two), dim))
    for p in range(n1):
        E[2 * p, p] = 1.0

    def put(x, y, z, col, c):
        # element of the antisymmetric spin-orbital tensor; like pair is (x, y) for IP, (y, z) for EA
        if kind == "ea":
            if y == z:
                return
            key, sgn = ((x, y, z), 1.0) if y < z else ((x, z, y), -1.0)
        else:
            if x == y:
                return
            key, sgn = ((x, y, z), 1.0) if x < y else ((y, x, z), -1.0)
        E[nso1 + pos[key], col] += sgn * c

    if kind == "ea":
        for i in range(o):
            for a in range(v):
                for b in range(v):
                    col = n1 + (i * v + a) * v + b
                    put(2 * i + 1, 2 * a + 1, 2 * b, col, 1.0)
                    put(2 * i, 2 * a, 2 * b, col, 0.5)
                    put(2 * i, 2 * b, 2 * a, col, -0.5)
    else:
        for j in range(o):
            for k in range(o):
                for a in range(v):
                    col = n1 + (j * o + k) * v + a
                    put(2 * j + 1, 2 * k, 2 * a + 1, col, 1.0)
                    put(2 * j, 2 * k, 2 * a, col, 0.5)
                    put(2 * k, 2 * j, 2 * a, col, -0.5)
    return E
