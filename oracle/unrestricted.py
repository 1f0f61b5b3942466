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
