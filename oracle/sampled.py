"""Sampled oracle outputs for sizes where the full tier-2 oracle is too slow.
TEST INFRASTRUCTURE ONLY -- nothing in the GPU product path may import this.

``sigma_ea_rows`` evaluates the EA-ADC(n) 2p1h rows sigma_{i,a,b} of the
spin-adapted sigma vector for a few chosen occupied indices i, from the same
working equations as ``spinadapted.SpinAdaptedADC`` (2p1h column of the
coupling block, zeroth-order diagonal, first-order ladder and ring terms), but
forming only the integral and amplitude slices that row i needs.  The 2p1h
rows do not depend on the 1p-1p block, so no O(o^2 v^4) setup is required.
It is pinned against the full tier-2 sigma in the CPU tests.
"""
from __future__ import annotations

import numpy as np

from .spinadapted import df_ladder


def sigma_ea_rows(eps, B, nocc, y1, Y2, rows, order=3):
    """sigma_{i,:,:} (EA, spin-adapted) for i in rows, for one trial vector.

    eps [nmo]; B [naux, nmo, nmo]; y1 [v] (1p part); Y2 [o, v, v] (2p1h part).
    Returns an array [len(rows), v, v].
    """
    o = nocc
    eps = np.asarray(eps, dtype=np.float64)
    eo, ev = eps[:o], eps[o:]
    Boo, Bov, Bvv = B[:, :o, :o], B[:, :o, o:], B[:, o:, o:]
    out = []
    # every term with a 1p factor is linear in y1: for y1 = 0 they vanish, and the full
    # amplitudes t_lm^ab (o^2 v^2) are not needed
    has1p = bool(np.any(y1))
    if order >= 3 and has1p:
        ovov = np.einsum("Qla,Qmb->lamb", Bov, Bov, optimize=True)
        D = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
        t = ovov.transpose(0, 2, 1, 3) / D  # t_lm^ab
        del ovov
    for i in rows:
        d = ev[:, None] + ev[None, :] - eo[i]
        s = d * Y2[i]
        if has1p:
            # (cb|ia) Y_c
            hq = np.einsum("Qcb,c->Qb", Bvv, y1, optimize=True)
            s = s + np.einsum("Qa,Qb->ab", Bov[:, i, :], hq, optimize=True)
        if order >= 3:
            if has1p:
                # amplitudes needed by row i: t_im^ae (all m) and t_lm^ba (all l, m)
                ovov_i = np.einsum("Qa,Qmb->amb", Bov[:, i, :], Bov, optimize=True)  # (ia|mb)
                t_i = ovov_i.transpose(1, 0, 2) / (eo[i] + eo[:, None, None] - ev[None, :, None] - ev[None, None, :])  # t_im^ab
                tau_i = 2.0 * t_i - t_i.transpose(0, 2, 1)
                # sum_lm (cl|im) t_lm^ba Y_c
                P = np.einsum("Qlc,c,Qm->lm", Bov, y1, Boo[:, i, :], optimize=True)
                s = s + np.einsum("lm,lmba->ab", P, t, optimize=True)
                # sum_me (cb|em) (2 t_im^ae - t_im^ea) Y_c
                q = np.einsum("Qb,Qme->bme", hq, Bov, optimize=True)
                s = s + np.einsum("bme,mae->ab", q, tau_i, optimize=True)
                # - sum_me (cm|eb) t_im^ae Y_c - sum_me (cm|ea) t_im^eb Y_c
                p = np.einsum("Qmc,c->Qm", Bov, y1, optimize=True)
                r = np.einsum("Qm,Qeb->meb", p, Bvv, optimize=True)
                s = s - np.einsum("meb,mae->ab", r, t_i, optimize=True)
                s = s - np.einsum("mea,meb->ab", r, t_i, optimize=True)
            # first-order 2p1h block: ladder and ring terms
            s = s + df_ladder(Bvv, Y2[i])
            oovv_i = np.einsum("Qj,Qac->jac", Boo[:, :, i], Bvv, optimize=True)  # (ji|ac)
            ovov_ij = np.einsum("Qa,Qjc->ajc", Bov[:, i, :], Bov, optimize=True)  # (ia|jc)
            s = s - np.einsum("jac,jcb->ab", oovv_i, Y2, optimize=True)
            s = s + 2.0 * np.einsum("ajc,jcb->ab", ovov_ij, Y2, optimize=True)
            s = s - np.einsum("ajc,jbc->ab", ovov_ij, Y2, optimize=True)
            s = s - np.einsum("jbd,jad->ab", oovv_i, Y2, optimize=True)
        out.append(s)
    return np.array(out)
