"""Training samples for the learned Davidson preconditioner (adc_mlp_train).

From a handle's own plain Davidson: the iterates y_k after k iterations (the
solver stopped at max_iter = k), their residuals r = sigma(y) - w y (adc_sigma)
and the exact correction t* = y_exact / <y, y_exact>_S - y, with y_exact the
tightly converged vector of the same root and S = diag(1, 2 - P) the metric
of the spin-adapted basis (Appendix).  Each sample is one vector element:
(d = D_x - w, blk = [x in the 1p/1h block], r_x, t*_x).
"""
from __future__ import annotations

import numpy as np


def _metric(x, o, v, kind):
    """S x for a vector of the spin-adapted layout (EA [v | o v v], IP [o | o o v])."""
    n1 = v if kind == "ea" else o
    y = x.copy()
    if kind == "ea":
        Y2 = x[n1:].reshape(o, v, v)
        y[n1:] = (2.0 * Y2 - Y2.transpose(0, 2, 1)).ravel()
    else:
        Y2 = x[n1:].reshape(o, o, v)
        y[n1:] = (2.0 * Y2 - Y2.transpose(1, 0, 2)).ravel()
    return y


def davidson_samples(adc, nroots, iters=(1, 2, 3, 4, 6, 8, 10, 14), per_vector=100_000, seed=0, exact_tol=1e-10):
    """(d, blk, r, t) sample arrays from the Davidson trajectory of `adc` (an ADC handle)."""
    o, v, kind = adc.nocc, adc.nvir, adc.kind
    dim = adc.dim
    n1 = v if kind == "ea" else o
    saved = dict(adc._solver)
    rng = np.random.default_rng(seed)
    D = adc.get("diag", (dim,))
    adc.set_options(max_iter=max(200, saved["max_iter"]), res_tol=min(1e-6, saved["res_tol"] or 1e-6))
    _, _, Yex, _ = adc.davidson(nroots, tol=exact_tol, want_vectors=True)
    SYex = np.array([_metric(y, o, v, kind) for y in Yex])
    out = [[], [], [], []]
    for k in iters:
        adc.set_options(max_iter=k, res_tol=1e-12)
        e, _, Y, _ = adc.davidson(nroots, tol=1e-14, want_vectors=True)
        W = adc.sigma(Y)
        for r in range(nroots):
            ov = SYex @ Y[r]  # <y_exact_s, y>_S for every exact root s
            s = int(np.argmax(np.abs(ov)))
            t = Yex[s] / ov[s] - Y[r]
            res = W[r] - e[r] * Y[r]
            pick = np.concatenate([np.arange(n1), n1 + rng.choice(dim - n1, min(per_vector, dim - n1), replace=False)])
            out[0].append(D[pick] - e[r])
            out[1].append((pick < n1).astype(np.uint8))
            out[2].append(res[pick])
            out[3].append(t[pick])
    adc.set_options(**saved)
    return tuple(np.concatenate(a) for a in out)
