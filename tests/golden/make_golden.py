"""Writes tests/golden/tier0_doublet_spectra.json from the tier-0 oracle only.

For tiny closed-shell systems the tier-0 (Fock-space, operator-definition)
oracle builds the full spin-orbital EA/IP-ADC(n) matrix (Eqs. M_ea, M_ip;
orders k+l+m = n, Sec. II A).  Its eigenvalues come in spin multiplets: each
doublet appears twice (M_S = +-1/2), each quartet four times.  The stored
values are the doublet eigenvalues -- the spectrum the spin-adapted code
(Sec. III B) must reproduce -- in the library's sign convention (EA:
eigenvalues of M_+; IP: eigenvalues of -M_-, the ionisation energies).

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from adc_inputs import make_system  # noqa: E402
from oracle.fock import ADCFock  # noqa: E402

SYSTEMS = [  # (nocc, nvir, naux, seed, scale of B)
    (2, 3, 10, 5, 2.0),
    (2, 4, 12, 8, 1.5),
]


def doublets(w, tol=1e-8):
    """Eigenvalues with multiplicity 2 (doublets), from a sorted spectrum."""
    w = np.sort(w)
    out, i = [], 0
    while i < len(w):
        j = i
        while j + 1 < len(w) and w[j + 1] - w[i] < tol:
            j += 1
        m = j - i + 1
        if m % 4 == 2:  # a doublet (possibly sharing its value with quartets)
            out.append(float(np.mean(w[i:j + 1])))
        elif m % 2:
            raise RuntimeError(f"odd multiplicity {m} at {w[i]}")
        i = j + 1
    return out


def main():
    cases = []
    for o, v, naux, seed, scale in SYSTEMS:
        s = make_system(o, v, naux, seed=seed)
        for order in (2, 3):
            F = ADCFock(s.eps, o, order, B=scale * s.B)
            for kind in ("ea", "ip"):
                mats, _ = F.adc_matrices(kind)
                M = sum(mats[k] for k in range(order + 1))  # M = M(0) + ... + M(n)
                w = np.linalg.eigvalsh(0.5 * (M + M.T))
                if kind == "ip":
                    w = -w
                cases.append({"nocc": o, "nvir": v, "naux": naux, "seed": seed, "B_scale": scale,
                              "order": order, "kind": kind, "doublets": doublets(w)})
    out = {"source": "oracle.fock.ADCFock (tier 0, operator definitions, Sec. II A Eqs. M_ea, M_ip)",
           "generator": "adc_inputs.make_system(nocc, nvir, naux, seed); B multiplied by B_scale",
           "convention": "EA: eigenvalues of M_+; IP: eigenvalues of -M_- (ionisation energies); doublets only",
           "cases": cases}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tier0_doublet_spectra.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, len(cases), "cases")


if __name__ == "__main__":
    main()
