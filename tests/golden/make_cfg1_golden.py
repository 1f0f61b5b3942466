"""Writes tests/golden/cfg1_roots.json from the oracle only (tier 2, spin-adapted
DF equations, FP64): the 5 lowest EA- and IP-ADC(3) roots and spectroscopic
factors of the synthetic system nocc=20, nvir=180, naux=600, seed 0 (the
plain-FP64 workload: Davidson tol 1e-8 Eh, <= 8 vectors per root), converged
here to |dw| <= 1e-10 and S-norm residual <= 1e-6.  Takes tens of minutes on
a CPU (the third-order 1p-1p block and ~300 sigma vectors of EA).

Run from the repository root:  python tests/golden/make_cfg1_golden.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from adc_inputs import make_system  # noqa: E402
from oracle.davidson import davidson, spectroscopic_factors  # noqa: E402
from oracle.spinadapted import SpinAdaptedADC  # noqa: E402


def main():
    o, v, naux, seed, nroots = 20, 180, 600, 0, 5
    s = make_system(o, v, naux, seed=seed)
    out = {"source": "oracle.spinadapted.SpinAdaptedADC + oracle.davidson.davidson (tier 2, FP64)",
           "system": {"nocc": o, "nvir": v, "naux": naux, "seed": seed, "order": 3},
           "convergence": {"tol": 1e-10, "res_tol": 1e-6, "max_space_per_root": 8}}
    for kind in ("ip", "ea"):
        t0 = time.time()
        T = SpinAdaptedADC(s.eps, o, s.B, 3, kind)
        w, Y, it, nsig = davidson(T, nroots, tol=1e-10, res_tol=1e-6, max_iter=400)
        P = spectroscopic_factors(T, Y)
        out[kind] = {"energies_eh": [float(x) for x in w], "spectroscopic_factors": [float(x) for x in P],
                     "iterations": int(it), "sigma_vectors": int(nsig), "seconds": time.time() - t0}
        print(kind, out[kind], flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg1_roots.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
