"""Eigen-solvers and spectroscopic factors for the spin-adapted oracle.
TEST INFRASTRUCTURE ONLY -- nothing in the GPU product path may import this.

* Eq. eig: M Y = Y Omega.  The spin-adapted matrix is S^-1 A with A = E^T M E
  symmetric and S = E^T E positive definite, so the problem is the symmetric-
  definite pencil A y = w S y.  ``dense_roots`` solves it directly (small
  systems); ``davidson`` is a plain multi-root Davidson iteration in the
  S inner product (the paper uses Davidson's method, Sec. III A, without giving
  its details; the readings used are listed in the function docstring).
* Spectroscopic factors (Appendix, Eqs. appendix_1..4): renormalise Y with the
  spin-adapted norm Y^T S Y, form X_p = sum_nu T_{p,nu} (S Y~)_nu and
  P = 2 sum_p X_p^2 (Eq. spec_factors with the factor 2 of the Appendix).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def dense_roots(adc, nroots):
    """Lowest nroots eigenpairs of the spin-adapted matrix (small systems)."""
    M = adc.dense()
    A = adc.apply_S(M.T).T  # S M
    A = 0.5 * (A + A.T)
    S = adc.apply_S(np.eye(adc.dim))
    w, Y = scipy.linalg.eigh(A, S)
    return w[:nroots], Y[:, :nroots].T


def transition_moments(adc, torder=None):
    """Spatial T through order n = torder, default adc.order (Eqs. T_ea, T_ip, k + l <= n):
    (T1 [nmo, n1], T2 [nmo, ...2p1h/2h1p shape]).

    Second order, with the density form B(x, y) (EA) / B'(x, y) (IP)
      B(x, y)_cb  = -sum x_kl^cd y_kl^bd + 1/2 sum x_kl^cd y_kl^db,
      B'(x, y)_kj = -sum x_kl^cd y_jl^cd + 1/2 sum x_kl^cd y_jl^dc:
    EA: T_{c,b} = d_cb + B(t, t)_cb, T_{k,b} = -t_k^b(2), T_{k,jcd} = -t_kj^dc, T_{c,jde} = 0.
    IP: T_{k,j} = d_kj + B'(t, t)_kj, T_{c,j} = t_j^c(2), T_{c,ija} = -t_ij^ac, T_{k,ija} = 0.
    (First order vanishes; t_k^b(2) enters M only at third order, so for
    ADC(2) it is still included here as the second-order T term.)
    Third order (ADC(3)) adds, with tau = 2t - t(ab swapped):
    EA: T_{c,b} += B(t, t2)_cb + B(t2, t)_cb, T_{k,b} -= t_k^b(3) + 1/2 sum tau_kl^bc t_l^c(2),
        T_{k,jcd} -= t2_kj^dc;
    IP: T_{k,j} += B'(t, t2)_kj + B'(t2, t)_kj, T_{c,j} += t_j^c(3) + 1/2 sum tau_jl^cd t_l^d(2),
        T_{c,ija} -= t2_ij^ac
    (t2 = t2(2); the spin integration of the spin-orbital third-order terms).
    """
    o, v = adc.o, adc.v
    t = adc.t
    t1 = adc.t1_2 if hasattr(adc, "t1_2") else _t1_second_order(adc)
    nmo = o + v
    third = (adc.order if torder is None else torder) >= 3 and adc.order >= 3
    if third:
        t2 = adc.t_2
        tau = 2.0 * t - t.transpose(0, 1, 3, 2)
    if adc.kind == "ea":
        def dens(x, y):
            return -np.einsum("klcd,klbd->cb", x, y) + 0.5 * np.einsum("klcd,kldb->cb", x, y)

        T1 = np.zeros((nmo, v))
        T1[o:] = np.eye(v) + dens(t, t)
        T1[:o] = -t1
        T2 = np.zeros((nmo, o, v, v))
        T2[:o] = -t.transpose(0, 1, 3, 2)
        if third:
            T1[o:] += dens(t, t2) + dens(t2, t)
            T1[:o] -= adc.t1_3 + 0.5 * np.einsum("klbc,lc->kb", tau, t1)
            T2[:o] -= t2.transpose(0, 1, 3, 2)
    else:
        def dens(x, y):
            return -np.einsum("klcd,jlcd->kj", x, y) + 0.5 * np.einsum("klcd,jldc->kj", x, y)

        T1 = np.zeros((nmo, o))
        T1[:o] = np.eye(o) + dens(t, t)
        T1[o:] = t1.T
        T2 = np.zeros((nmo, o, o, v))
        T2[o:] = -t.transpose(3, 0, 1, 2)
        if third:
            T1[:o] += dens(t, t2) + dens(t2, t)
            T1[o:] += adc.t1_3.T + 0.5 * np.einsum("jlcd,ld->cj", tau, t1)
            T2[o:] -= t2.transpose(3, 0, 1, 2)
    return T1, T2


def _t1_second_order(adc):
    tau = 2.0 * adc.t - adc.t.transpose(0, 1, 3, 2)
    s1 = np.einsum("Qkc,Qad,ikdc->ia", adc.Bov, adc.Bvv, tau, optimize=True)
    s2 = np.einsum("kilc,klac->ia", adc.ooov, tau)
    return (s1 - s2) / adc.D1


def spectroscopic_factors(adc, Y, torder=None):
    """P for each row of Y[nroots, dim] (Appendix normalisation), T through order torder (default n)."""
    Y = np.atleast_2d(Y)
    T1, T2 = transition_moments(adc, torder)
    SY = adc.apply_S(Y)
    norm = np.einsum("rk,rk->r", Y, SY)
    Yt = SY / np.sqrt(norm)[:, None]
    n1 = adc.n1
    X = Yt[:, :n1] @ T1.T + Yt[:, n1:] @ T2.reshape(T2.shape[0], -1).T
    return 2.0 * np.einsum("rp,rp->r", X, X)


def davidson(adc, nroots, tol=1e-8, max_space_per_root=8, max_iter=200, nguess_extra=2, guess=None, keep_per_root=2,
             res_tol=None):
    """Multi-root Davidson in the S inner product, FP64, diagonal preconditioner.

    Readings (the paper does not give them): guesses are unit vectors at the
    nroots + nguess_extra lowest diagonal elements (diag(M_11) and the zeroth-
    order 2p1h/2h1p energies); correction t = r / (w - D) with |w - D| kept
    >= 1e-8; a root is converged when |dw| <= tol and ||r||_S <= sqrt(tol);
    the space is collapsed to the lowest keep_per_root * nroots Ritz vectors
    when it would exceed max_space_per_root * nroots (res_tol, if given,
    replaces sqrt(tol)).
    Returns (w[nroots], Y[nroots, dim], n_iterations, n_sigma).
    """
    dim = adc.dim
    D = adc.diagonal()
    nstart = min(dim, nroots + nguess_extra)
    if guess is None:
        idx = np.argsort(D, kind="stable")[:nstart]
        V = np.zeros((nstart, dim))
        V[np.arange(nstart), idx] = 1.0
    else:
        V = np.array(guess, dtype=float)
    V = _s_orthonormalise(adc, V, np.zeros((0, dim)))
    W = adc.sigma(V)
    nsig = V.shape[0]
    w_old = np.full(nroots, np.inf)
    maxspace = max(max_space_per_root * nroots, max(nstart, keep_per_root * nroots) + nroots)
    rtol = np.sqrt(tol) if res_tol is None else res_tol
    for it in range(1, max_iter + 1):
        G = V @ adc.apply_S(W).T
        G = 0.5 * (G + G.T)
        e_all, C_all = np.linalg.eigh(G)
        e, C = e_all[:nroots], C_all[:, :nroots]
        X = C.T @ V
        AX = C.T @ W
        R = AX - e[:, None] * X
        rnorm = np.sqrt(np.einsum("rk,rk->r", R, adc.apply_S(R)))
        conv = (np.abs(e - w_old) <= tol) & (rnorm <= rtol)
        w_old = e
        if np.all(conv):
            return e, X, it, nsig
        new = []
        for r in range(nroots):
            if conv[r]:
                continue
            den = e[r] - D
            den = np.where(np.abs(den) < 1e-8, np.copysign(1e-8, den), den)
            new.append(R[r] / den)
        new = np.array(new)
        if V.shape[0] + new.shape[0] > maxspace:
            nkeep = min(V.shape[0], keep_per_root * nroots)
            Ck = C_all[:, :nkeep]
            V, W = Ck.T @ V, Ck.T @ W  # Ritz vectors are S-orthonormal; W stays sigma(V)
        new = _s_orthonormalise(adc, new, V)
        if new.shape[0] == 0:
            return e, X, it, nsig
        Wn = adc.sigma(new)
        nsig += new.shape[0]
        V = np.concatenate([V, new])
        W = np.concatenate([W, Wn])
    raise RuntimeError("Davidson did not converge")


def _s_orthonormalise(adc, new, V, drop=1e-10):
    out = []
    basis = [v for v in V]
    for x in new:
        x = x.copy()
        for _ in range(2):
            for b in basis + out:
                x -= (b @ adc.apply_S(x)) * b
        n = np.sqrt(x @ adc.apply_S(x))
        if n > drop:
            out.append(x / n)
    return np.array(out) if out else np.zeros((0, new.shape[1]))
