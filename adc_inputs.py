"""Seeded synthetic inputs for density-fitted EA/IP-ADC(n).

This module only draws random numbers; it holds none of the method's arithmetic.
Both the CPU oracle (``oracle/``) and the GPU path's tests and benchmark take
their inputs from here, so that the two sides see identical data.

Recipe (stands in for the paper's molecules, whose orbitals and integrals are
not available; shapes follow the paper's workloads up to 1028 orbitals):

* occupied orbital energies  eps_occ ~ U[-1.5, -0.3] Eh, sorted ascending;
* virtual orbital energies   eps_vir = 0.05 + U[0,1]**2 * 4.95 Eh, sorted;
* density-fitting factors    B^Q_pq = s (G + G^T)/2 with G ~ N(0,1) and
  s = 0.3 / sqrt(naux), so that (pq|rs) ~ sum_Q B^Q_pq B^Q_rs (Sec. III C,
  Eq. 19) has O(0.1) magnitude;
* draw order is fixed: eps_occ, eps_vir, then G one auxiliary index Q at a
  time (Q-major), all from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class System:
    nocc: int
    nvir: int
    naux: int
    eps: np.ndarray  # [nmo] float64, occupied first, each block ascending
    B: np.ndarray  # [naux, nmo, nmo] float64, symmetric in the last two indices

    @property
    def nmo(self) -> int:
        return self.nocc + self.nvir


def make_system(nocc: int, nvir: int, naux: int, seed: int = 0, dtype=np.float64) -> System:
    """Draw one synthetic closed-shell system (see the module docstring)."""
    rng = np.random.default_rng(seed)
    eps_o = np.sort(rng.uniform(-1.5, -0.3, size=nocc))
    eps_v = np.sort(0.05 + rng.uniform(0.0, 1.0, size=nvir) ** 2 * 4.95)
    nmo = nocc + nvir
    s = 0.3 / np.sqrt(naux)
    B = np.empty((naux, nmo, nmo), dtype=dtype)
    for q in range(naux):
        g = rng.standard_normal((nmo, nmo))
        B[q] = (s * 0.5) * (g + g.T)
    return System(nocc, nvir, naux, np.concatenate([eps_o, eps_v]), B)


def make_trial_vectors(dim: int, nvec: int, seed: int = 1) -> np.ndarray:
    """Random trial vectors X[nvec, dim] ~ N(0,1) / sqrt(dim) (for sigma parity tests)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nvec, dim)) / np.sqrt(dim)


def make_psd_eri(nmo: int, seed: int = 3, scale: float = 0.05) -> np.ndarray:
    """A random positive semi-definite two-electron tensor (pq|rs) with 8-fold symmetry.

    Built as W^T W over the symmetric pair space, so it has an exact
    factorisation with naux = nmo (nmo + 1) / 2 (used to check that density
    fitting with a complete auxiliary set reproduces the four-index result).
    """
    rng = np.random.default_rng(seed)
    npair = nmo * (nmo + 1) // 2
    W = rng.standard_normal((npair, npair)) * scale / np.sqrt(npair)
    G = W.T @ W
    iu = np.triu_indices(nmo)
    pair = np.zeros((nmo, nmo), dtype=np.int64)
    pair[iu] = np.arange(npair)
    pair[(iu[1], iu[0])] = np.arange(npair)
    return G[pair[:, :, None, None], pair[None, None, :, :]]


@dataclasses.dataclass
class OpenShellSystem:
    nocc_a: int
    nocc_b: int
    eps_a: np.ndarray  # [nmo] alpha orbital energies, occupied first, each block ascending
    eps_b: np.ndarray  # [nmo] beta orbital energies
    B_a: np.ndarray  # [naux, nmo, nmo] alpha-orbital DF factors, symmetric in the last two indices
    B_b: np.ndarray  # [naux, nmo, nmo] beta-orbital DF factors

    @property
    def nmo(self) -> int:
        return len(self.eps_a)


def make_open_shell_system(nocc_a: int, nocc_b: int, nmo: int, naux: int, seed: int = 0) -> OpenShellSystem:
    """Synthetic unrestricted (open-shell) reference: alpha and beta orbitals
    share one auxiliary-basis tensor b^Q (drawn as in make_system) but have
    their own orthonormal orbital coefficients C_s = Q factor of
    (1 + 0.2 N(0,1)), so that B_s^Q = C_s^T b^Q C_s; orbital energies are drawn
    per spin as in make_system with nocc_a / nocc_b occupied.  Draw order:
    eps (alpha occ, alpha vir, beta occ, beta vir), b^Q (Q-major), C_a, C_b."""
    rng = np.random.default_rng(seed)

    def energies(no):
        return np.concatenate([np.sort(rng.uniform(-1.5, -0.3, size=no)),
                               np.sort(0.05 + rng.uniform(0.0, 1.0, size=nmo - no) ** 2 * 4.95)])

    eps_a, eps_b = energies(nocc_a), energies(nocc_b)
    s = 0.3 / np.sqrt(naux)
    b = np.empty((naux, nmo, nmo))
    for q in range(naux):
        g = rng.standard_normal((nmo, nmo))
        b[q] = (s * 0.5) * (g + g.T)
    C = []
    for _ in range(2):
        Cq, _r = np.linalg.qr(np.eye(nmo) + 0.2 * rng.standard_normal((nmo, nmo)))
        C.append(Cq)
    B_a = np.einsum("pm,Qpq,qn->Qmn", C[0], b, C[0])
    B_b = np.einsum("pm,Qpq,qn->Qmn", C[1], b, C[1])
    return OpenShellSystem(nocc_a, nocc_b, eps_a, eps_b, B_a, B_b)


# Named workloads (sizes of the paper-shaped synthetic cases).
CONFIGS = {
    "ea2_small": dict(nocc=5, nvir=20, naux=80, order=2, kind="ea", nroots=4),
    "adc3_medium": dict(nocc=20, nvir=180, naux=600, order=3, nroots=5),
    "ea3_large": dict(nocc=40, nvir=400, naux=1400, order=3, kind="ea", nroots=4),
    "ea3_huge": dict(nocc=68, nvir=960, naux=3000, order=3, kind="ea", nroots=4),
}


def batched_ip_molecules(nmol: int = 64):
    """Sizes of the batched IP workload: nocc ~ U{8..30}, nvir ~ U{60..250},
    naux = round(3.5 (nocc + nvir)), seeds 0..nmol-1."""
    out = []
    for seed in range(nmol):
        rng = np.random.default_rng(10_000 + seed)
        o = int(rng.integers(8, 31))
        v = int(rng.integers(60, 251))
        out.append(dict(nocc=o, nvir=v, naux=int(round(3.5 * (o + v))), seed=seed))
    return out
