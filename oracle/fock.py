"""Tier-0 oracle: EA/IP-ADC(n) matrices from their operator definitions, by
brute force in Fock space.  TEST INFRASTRUCTURE ONLY -- nothing in the GPU
product path may import this module.

What it follows, step by step (Sec. II A of the paper):

* H = H(0) + V.  H(0) = sum_p eps_p {p+ p} (diagonal Fock operator, Moller--
  Plesset partitioning) and V is the normal-ordered two-electron operator built
  from <pq||rs> = (pr|qs) - (ps|qr) with (pq|rs) = sum_Q B^Q_pq B^Q_rs (Eq. 19).
  Synthetic eps and B are not self-consistent, so the reading used here is
  that the Fock operator *is* diag(eps): the mean-field one-body part of the
  bare two-electron operator is removed together with its constant.
* Unitary ground state exp(T - T+) Phi (Eq. gs_wavefunction) with T = T1 + T2
  (Eq. ex_op).  Amplitudes are found order by order from the singles and
  doubles projections of the k-th order effective Hamiltonian (Eqs.
  t_singles, t_doubles): singles up to order n, doubles up to order n-1.
* Effective Hamiltonian and observable by the BCH series (Eqs. H_bch,
  ap_bch), collected order by order.
* M^(n)_{mu nu} = sum_{k+l+m=n} <Phi|{h_mu^(k), [Ht^(l), h_nu^(m)+]}|Phi>
  (Eqs. M_ea, M_ip) and T^(n)_{p nu} = sum_{k+l=n} <Phi|{a~_p^(k),
  h_nu^(l)+}|Phi> (Eqs. T_ea, T_ip), with h+ = a_a+, a_b+ a_a+ a_i (EA) and
  h+ = a_i, a_a+ a_j a_i (IP) as the paper lists them.

Conventions: spin orbital P = 2 p + s (s = 0 alpha, 1 beta), spatial orbitals
occupied first.  Operators that conserve the particle number are dense
matrices on one N-electron sector at a time.  Feasible up to ~14 spin orbitals.

Sign convention for IP: the matrix returned is the paper's M_- (eigenvalues
E_N - E_{N-1}); callers that want ionisation energies negate it.
"""
from __future__ import annotations

import math
from itertools import combinations

import numpy as np
import scipy.sparse as sp


def _popcount(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.int64)
    c = np.zeros_like(x)
    while np.any(x):
        c += x & 1
        x = x >> 1
    return c


class FockSpace:
    """Determinants of nso spin orbitals, grouped by particle number."""

    def __init__(self, nso: int):
        self.nso = nso
        self.dets = {}
        self.index = {}
        for n in range(nso + 1):
            d = np.array(sorted(sum(1 << p for p in c) for c in combinations(range(nso), n)), dtype=np.int64)
            self.dets[n] = d
            self.index[n] = {int(v): i for i, v in enumerate(d)}

    def dim(self, n):
        return len(self.dets[n])

    def apply_string(self, ops, n):
        """Matrix of an operator string acting on sector n.

        ops is a list of (P, dagger) in the order they are written (leftmost
        first); the rightmost acts first.  Returns (rows, cols, signs, n_out).
        """
        dets = self.dets[n].copy()
        sign = np.ones(len(dets), dtype=np.int64)
        ok = np.ones(len(dets), dtype=bool)
        nout = n
        for P, dag in reversed(ops):
            bit = np.int64(1) << np.int64(P)
            occ = (dets & bit) != 0
            ok &= (~occ) if dag else occ
            below = _popcount(dets & (bit - 1))
            sign *= np.where(below % 2 == 0, 1, -1)
            dets = dets ^ bit
            nout += 1 if dag else -1
        cols = np.nonzero(ok)[0]
        if nout < 0 or nout > self.nso:
            return np.array([], dtype=np.int64), cols[:0], sign[:0], nout
        rows = np.searchsorted(self.dets[nout], dets[cols]).astype(np.int64)
        return rows, cols, sign[cols], nout

    def string_matrix(self, ops, n, coeff=1.0):
        rows, cols, sgn, nout = self.apply_string(ops, n)
        m = sp.csr_matrix((coeff * sgn.astype(float), (rows, cols)), shape=(self.dim(nout), self.dim(n)))
        return m, nout

    def op_sum_dense(self, terms, n):
        """Dense matrix on sector n (-> same sector) of sum_k c_k * string_k."""
        M = np.zeros((self.dim(n), self.dim(n)))
        for c, ops in terms:
            if c == 0.0:
                continue
            rows, cols, sgn, nout = self.apply_string(ops, n)
            assert nout == n
            np.add.at(M, (rows, cols), c * sgn)
        return M


def spin_orbital_integrals(B: np.ndarray):
    """<PQ||RS> for spin orbitals P = 2p+s from spatial (pq|rs) = sum_Q B^Q_pq B^Q_rs."""
    eri = np.einsum("Qpq,Qrs->pqrs", B, B)
    return spin_orbital_antisym(eri)


def spin_orbital_antisym(eri: np.ndarray) -> np.ndarray:
    nmo = eri.shape[0]
    nso = 2 * nmo
    spin = np.arange(nso) % 2
    sp_ = np.arange(nso) // 2
    # <PQ|RS> = (PR|QS) delta(sP,sR) delta(sQ,sS)
    phys = eri[sp_[:, None, None, None], sp_[None, None, :, None], sp_[None, :, None, None], sp_[None, None, None, :]]
    mask = (spin[:, None, None, None] == spin[None, None, :, None]) & (spin[None, :, None, None] == spin[None, None, None, :])
    phys = phys * mask
    return phys - phys.transpose(0, 1, 3, 2)


class ADCFock:
    """Brute-force EA/IP-ADC(n) for a tiny closed-shell system.

    eps: spatial orbital energies [nmo] (occupied first); either B [naux, nmo,
    nmo] or eri [nmo]*4 (chemists' notation, spatial) defines the integrals.
    """

    def __init__(self, eps, nocc, order, B=None, eri=None):
        eps = np.asarray(eps, dtype=float)
        if eri is None:
            eri = np.einsum("Qpq,Qrs->pqrs", B, B)
        self._init_spin_orbitals(np.repeat(eps, 2), 2 * nocc, spin_orbital_antisym(np.asarray(eri, dtype=float)), order)

    @classmethod
    def from_spin_orbitals(cls, eps_so, no, asym, order):
        """Any reference given in spin orbitals: energies eps_so [nso], the
        first `no` spin orbitals occupied, antisymmetrised <PQ||RS> [nso]^4
        (unrestricted open-shell references, Sec. II)."""
        self = cls.__new__(cls)
        self._init_spin_orbitals(np.asarray(eps_so, dtype=float), no, np.asarray(asym, dtype=float), order)
        return self

    def _init_spin_orbitals(self, eps_so, no, asym, order):
        self.order = order
        self.nso = len(eps_so)
        self.no = no
        self.eps_so = eps_so
        self.asym = asym
        self.fs = FockSpace(self.nso)
        self.N = self.no
        self.occ = list(range(self.no))
        self.vir = list(range(self.no, self.nso))
        self.phi = self.fs.index[self.N][(1 << self.no) - 1]
        self.sectors = [self.N - 1, self.N, self.N + 1]
        self._build_hamiltonian()
        self._solve_amplitudes()
        self._effective_hamiltonian()

    # -- Hamiltonian -----------------------------------------------------
    def _h0_terms(self):
        n = np.zeros(self.nso)
        n[: self.no] = 1.0
        return [(self.eps_so[P], [(P, True), (P, False)]) for P in range(self.nso)], float(-(self.eps_so * n).sum())

    def _v_terms(self):
        """Normal-ordered V: bare 1/4 <pq||rs> p+q+sr, minus mean field, plus constant."""
        A = self.asym
        terms = []
        nso = self.nso
        for p, q in combinations(range(nso), 2):
            for r, s in combinations(range(nso), 2):
                c = A[p, q, r, s]
                if abs(c) > 0.0:
                    terms.append((c, [(p, True), (q, True), (s, False), (r, False)]))
        occ = self.occ
        fmf = np.einsum("pioi->po", A[:, occ][:, :, :, occ])
        for p in range(nso):
            for q in range(nso):
                if abs(fmf[p, q]) > 0.0:
                    terms.append((-fmf[p, q], [(p, True), (q, False)]))
        const = 0.5 * sum(A[i, j, i, j] for i in occ for j in occ)
        return terms, const

    def _build_hamiltonian(self):
        h0t, h0c = self._h0_terms()
        vt, vc = self._v_terms()
        self.H0 = {}
        self.V = {}
        for n in self.sectors:
            I = np.eye(self.fs.dim(n))
            self.H0[n] = self.fs.op_sum_dense(h0t, n) + h0c * I
            self.V[n] = self.fs.op_sum_dense(vt, n) + vc * I

    # -- amplitudes --------------------------------------------------------
    def _singles(self):
        return [(i, a) for i in self.occ for a in self.vir]

    def _doubles(self):
        return [(i, j, a, b) for i, j in combinations(self.occ, 2) for a, b in combinations(self.vir, 2)]

    def _exc_strings(self):
        S = [[(a, True), (i, False)] for i, a in self._singles()]
        D = [[(a, True), (b, True), (j, False), (i, False)] for i, j, a, b in self._doubles()]
        return S, D

    def _sigma_from_amplitudes(self, t1, t2):
        """sigma = T - T+ on every sector, T = sum t1 a+i + sum_{i<j,a<b} t2 a+b+ji."""
        S, D = self._exc_strings()
        terms = [(c, s) for c, s in zip(t1, S)] + [(c, s) for c, s in zip(t2, D)]
        out = {}
        for n in self.sectors:
            T = self.fs.op_sum_dense(terms, n)
            out[n] = T - T.T
        return out

    def _bch_orders(self, sig_by_order, nmax):
        """C[k][m] = order-m part of ad^k(H); returns Ht[m] = sum_k C[k][m]/k!, m<=nmax."""
        Ht = {}
        for n in self.sectors:
            C = [{0: self.H0[n], 1: self.V[n]}]
            for k in range(1, nmax + 1):
                ck = {}
                for m in range(k, nmax + 1):
                    acc = None
                    for mm, sig in sig_by_order.items():
                        prev = C[k - 1].get(m - mm)
                        if prev is None or mm < 1:
                            continue
                        s = sig[n]
                        term = prev @ s - s @ prev
                        acc = term if acc is None else acc + term
                    if acc is not None:
                        ck[m] = acc
                C.append(ck)
            for m in range(nmax + 1):
                acc = np.zeros_like(self.H0[n])
                for k in range(len(C)):
                    if m in C[k]:
                        acc = acc + C[k][m] / math.factorial(k)
                Ht.setdefault(m, {})[n] = acc
        return Ht

    def _solve_amplitudes(self):
        nmax = self.order
        S, D = self._exc_strings()
        singles, doubles = self._singles(), self._doubles()
        e = self.eps_so
        Ds = np.array([e[i] - e[a] for i, a in singles])
        Dd = np.array([e[i] + e[j] - e[a] - e[b] for i, j, a, b in doubles])
        N = self.N
        phi = np.zeros(self.fs.dim(N))
        phi[self.phi] = 1.0
        self.phi_vec = phi
        # projection vectors <Phi_mu| in sector N
        Pv_s = [self.fs.string_matrix(s, N)[0] @ phi for s in S]
        Pv_d = [self.fs.string_matrix(s, N)[0] @ phi for s in D]
        self.t1 = {}
        self.t2 = {}
        sig = {}
        for k in range(1, nmax + 1):
            Ht = self._bch_orders(sig, k)
            R = Ht[k][N] @ phi
            t1 = np.array([v @ R for v in Pv_s]) / Ds
            t2 = np.array([v @ R for v in Pv_d]) / Dd
            if k > nmax - 1:  # doubles only up to order n-1
                t2 = np.zeros_like(t2)
            self.t1[k] = t1
            self.t2[k] = t2
            sig[k] = self._sigma_from_amplitudes(t1, t2)
        self.sig = sig

    def _effective_hamiltonian(self):
        self.Ht = self._bch_orders(self.sig, self.order)

    # -- amplitude tensors for comparisons --------------------------------
    def t1_tensor(self, k):
        no, nv = self.no, self.nso - self.no
        out = np.zeros((no, nv))
        for c, (i, a) in zip(self.t1[k], self._singles()):
            out[i, a - no] = c
        return out

    def t2_tensor(self, k):
        no, nv = self.no, self.nso - self.no
        out = np.zeros((no, no, nv, nv))
        for c, (i, j, a, b) in zip(self.t2[k], self._doubles()):
            a -= no
            b -= no
            out[i, j, a, b] = c
            out[j, i, a, b] = -c
            out[i, j, b, a] = -c
            out[j, i, b, a] = c
        return out

    def energy(self, k):
        """k-th order contribution to the ground-state energy <Phi|Ht^(k)|Phi>."""
        return float(self.phi_vec @ self.Ht[k][self.N] @ self.phi_vec)

    # -- ADC basis ----------------------------------------------------------
    def basis(self, kind):
        """Basis operators A_mu (annihilation type) with order labels.

        EA: A = h_mu: a_a (order 0) and (a_b+ a_a+ a_i)+ = a_i+ a_a a_b (order 1), a<b.
        IP: A = h_-mu+: a_i (order 0) and a_a+ a_j a_i (order 1), i<j.
        Returned as lists of (label, order, string of A_mu).
        """
        out = []
        if kind == "ea":
            for a in self.vir:
                out.append((("p", a), 0, [(a, False)]))
            for i in self.occ:
                for a, b in combinations(self.vir, 2):
                    out.append((("pph", i, a, b), 1, [(i, True), (a, False), (b, False)]))
        else:
            for i in self.occ:
                out.append((("h", i), 0, [(i, False)]))
            for a in self.vir:
                for i, j in combinations(self.occ, 2):
                    out.append((("hhp", i, j, a), 1, [(a, True), (j, False), (i, False)]))
        return out

    @staticmethod
    def _adjoint(ops):
        return [(P, not d) for P, d in reversed(ops)]

    def adc_pieces(self, kind):
        """<Phi|{A_mu, [Ht^(l), A_nu+]}|Phi> for every basis pair and l = 0..order.

        Returns ({l: matrix}, basis, order labels).  M^(n) keeps, for the pair
        (mu, nu), the piece with l = n - k_mu - k_nu (k = operator order label).
        """
        bas = self.basis(kind)
        N = self.N
        fs = self.fs
        phi = self.phi_vec
        nb = len(bas)
        # u_nu = A_nu+ |Phi> (sector N+1), w_nu = A_nu |Phi> (sector N-1)
        U = np.zeros((nb, fs.dim(N + 1)))
        W = np.zeros((nb, fs.dim(N - 1)))
        Adag_lo = []  # A_nu+ : N-1 -> N
        Adag_mid = []  # A_nu+ : N -> N+1
        for k, (_, _, s) in enumerate(bas):
            sd = self._adjoint(s)
            m_mid, nout = fs.string_matrix(sd, N)
            U[k] = m_mid @ phi
            m_lo, _ = fs.string_matrix(sd, N - 1)
            Adag_mid.append(m_mid)
            Adag_lo.append(m_lo)
            m_a, _ = fs.string_matrix(s, N)
            W[k] = m_a @ phi
        orders = np.array([o for _, o, _ in bas])
        pieces = {}
        for l in range(self.order + 1):
            H = self.Ht[l]
            hphi = H[N] @ phi
            t1 = U @ H[N + 1] @ U.T  # <Phi|A_mu H A_nu+|Phi>
            AH = np.stack([Adag_mid[nu] @ hphi for nu in range(nb)], axis=1)  # [dim N+1, nb]
            t2 = U @ AH  # <Phi|A_mu A_nu+ H|Phi>
            AW = np.stack([hphi @ Adag_lo[nu] for nu in range(nb)], axis=0)  # [nb, dim N-1]
            t3 = (AW @ W.T).T  # <Phi|H A_nu+ A_mu|Phi>
            t4 = W @ H[N - 1] @ W.T  # [nu', mu'] -> <Phi|A_nu'+ H A_mu'|Phi>
            pieces[l] = t1 - t2 + t3 - t4.T
        return pieces, bas, orders

    def adc_matrices(self, kind):
        """M^(n) for n = 0..order (dict) in the basis of `basis(kind)`."""
        pieces, bas, orders = self.adc_pieces(kind)
        out = {}
        for n in range(self.order + 1):
            M = np.zeros_like(pieces[0])
            for l in range(n + 1):
                sel = (orders[:, None] + orders[None, :] + l) == n
                M += np.where(sel, pieces[l], 0.0)
            out[n] = M
        return out, bas

    def _dressed_annihilators(self, nmax):
        """a~_p^(k): list over k of {n: matrix sector n -> n-1} for each spin orbital p."""
        res = []
        for p in range(self.nso):
            per = {}
            for n in (self.N, self.N + 1):
                a, _ = self.fs.string_matrix([(p, False)], n)
                a = a.toarray()
                C = [{0: a}]
                for k in range(1, nmax + 1):
                    ck = {}
                    for m in range(k, nmax + 1):
                        acc = None
                        for mm, sig in self.sig.items():
                            prev = C[k - 1].get(m - mm)
                            if prev is None:
                                continue
                            term = prev @ sig[n] - sig[n - 1] @ prev
                            acc = term if acc is None else acc + term
                        if acc is not None:
                            ck[m] = acc
                    C.append(ck)
                ords = {}
                for m in range(nmax + 1):
                    acc = np.zeros_like(a)
                    for k in range(len(C)):
                        if m in C[k]:
                            acc = acc + C[k][m] / math.factorial(k)
                    ords[m] = acc
                per[n] = ords
            res.append(per)
        return res

    def adc_transition(self, kind, torder=None):
        """T^(n)_{p nu} for n = 0..torder (dict of [nso, nbasis])."""
        torder = self.order if torder is None else torder
        bas = self.basis(kind)
        N = self.N
        fs = self.fs
        phi = self.phi_vec
        at = self._dressed_annihilators(torder)
        out = {n: np.zeros((self.nso, len(bas))) for n in range(torder + 1)}
        for nu, (_, o, s) in enumerate(bas):
            sd = self._adjoint(s)
            m_mid, _ = fs.string_matrix(sd, N)  # N -> N+1
            m_lo, _ = fs.string_matrix(sd, N - 1)  # N-1 -> N
            u = m_mid @ phi
            for p in range(self.nso):
                for k in range(torder + 1 - o):
                    val = phi @ (at[p][N + 1][k] @ u) + phi @ (m_lo @ (at[p][N][k] @ phi))
                    out[k + o][p, nu] += val
        return out, bas
