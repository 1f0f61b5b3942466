"""ctypes binding of libadc.so: argument marshalling only (see include/adc.h)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "_build", "libadc.so")
_lib = None

ADC_OK, ADC_ERR_ARG, ADC_ERR_OOM, ADC_ERR_CUDA, ADC_ERR_NOT_CONVERGED, ADC_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
ADC_EA, ADC_IP = 1, -1
PRECISIONS = {"fp64": 0, "bf16x3": 1}

EXPORTED = [
    "adc_set_options",
    "adc_mlp_nweights",
    "adc_mlp_loss_grad",
    "adc_mlp_train",
    "adc_set_mlp",
    "adc_mlp_nsamples",
    "adc_mlp_samples",
    "adc_spectrum",
    "adc_setup_batch",
    "adc_davidson_batch",
    "adc_default_options",
    "adc_setup",
    "adc_dim",
    "adc_set_stream",
    "adc_sigma",
    "adc_davidson",
    "adc_get_tensor",
    "adc_mp_energy",
    "adc_setup_unrestricted",
    "adc_kernel_timing",
    "adc_kernel_launches",
    "adc_ladder_noalloc",
    "adc_last_error",
    "adc_destroy",
]


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("max_space_per_root", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("nguess_extra", ctypes.c_int),
        ("res_tol", ctypes.c_double),
        ("aux_chunk", ctypes.c_int),
        ("keep_per_root", ctypes.c_int),
        ("contractions", ctypes.c_int),
        ("refine", ctypes.c_int),
        ("transition_order", ctypes.c_int),
        ("refine_res_tol", ctypes.c_double),
        ("m11_on_the_fly", ctypes.c_int),
        ("tune_cache", ctypes.c_char_p),
        ("cuda_graphs", ctypes.c_int),
        ("lean", ctypes.c_int),
    ]


class ADCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def library_path() -> str:
    return _LIBPATH


def build_library(verbose: bool = False) -> str:
    from .build import build

    return build(verbose=verbose)


def load_library():
    """Load libadc.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIBPATH):
        raise ImportError(f"libadc.so not built at {_LIBPATH}; run __graft_entry__.build()")
    lib = ctypes.CDLL(_LIBPATH)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    lib.adc_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.adc_setup.argtypes = [P, P, I, I, I, I, I, ctypes.POINTER(Options), I, ctypes.POINTER(P)]
    lib.adc_dim.argtypes = [P, ctypes.POINTER(LL)]
    lib.adc_set_stream.argtypes = [P, P]
    lib.adc_sigma.argtypes = [P, P, P, I, I]
    lib.adc_davidson.argtypes = [P, I, D, P, P, P, P, P]
    lib.adc_get_tensor.argtypes = [P, ctypes.c_char_p, P, LL]
    lib.adc_mp_energy.argtypes = [P, P, ctypes.c_int]
    lib.adc_setup_unrestricted.argtypes = [P, P, P, P, I, I, I, I, I, I, ctypes.POINTER(Options), ctypes.POINTER(P)]
    lib.adc_kernel_timing.argtypes = [P, I, P]
    lib.adc_kernel_launches.argtypes = [P, P, LL]
    lib.adc_kernel_launches.restype = LL
    lib.adc_ladder_noalloc.argtypes = [P, P, P, LL]
    lib.adc_spectrum.argtypes = [P, P, I, D, P, I, P]
    lib.adc_mlp_nweights.argtypes = []
    lib.adc_mlp_loss_grad.argtypes = [P, P, P, P, P, LL, P, P]
    lib.adc_mlp_train.argtypes = [P, P, P, P, P, LL, I, ctypes.c_float, P]
    lib.adc_set_mlp.argtypes = [P, P]
    lib.adc_mlp_nsamples.argtypes = [P, I, I, LL]
    lib.adc_mlp_nsamples.restype = LL
    lib.adc_mlp_samples.argtypes = [P, I, P, I, LL, ctypes.c_ulonglong, D, P, P, P, P, LL]
    lib.adc_set_options.argtypes = [P, ctypes.POINTER(Options)]
    lib.adc_setup_batch.argtypes = [I, P, P, P, P, P, I, I, ctypes.POINTER(Options), I, P]
    lib.adc_davidson_batch.argtypes = [P, I, I, D, P, P, P, P]
    lib.adc_last_error.argtypes = [P]
    lib.adc_last_error.restype = ctypes.c_char_p
    lib.adc_destroy.argtypes = [P]
    lib.adc_destroy.restype = None
    for name in EXPORTED:
        if not hasattr(lib, name):
            raise ImportError(f"libadc.so lacks {name}")
    _lib = lib
    return lib


def spectrum(energies, specfac, omega, eta):
    """A(omega) of computed roots (Eqs. spec_function, PES) through adc_spectrum."""
    lib = load_library()
    e = np.ascontiguousarray(energies, dtype=np.float64)
    p = np.ascontiguousarray(specfac, dtype=np.float64)
    w = np.ascontiguousarray(omega, dtype=np.float64)
    if e.shape != p.shape:
        raise ValueError("energies and specfac differ in length")
    out = np.zeros(w.shape)
    rc = lib.adc_spectrum(e.ctypes.data, p.ctypes.data, e.size, float(eta), w.ctypes.data, w.size, out.ctypes.data)
    if rc != ADC_OK:
        raise ADCError(rc, "adc_spectrum: invalid argument")
    return out


def _ptr(a):
    """(pointer, on_device) for a numpy array or a CUDA torch tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data, 0
    return a.data_ptr(), 1


class ADC:
    """One system: setup on construction, then sigma / davidson.

    eps [nmo] and B [naux, nmo, nmo] are float64 numpy arrays (host) or CUDA
    torch tensors (device); kind 'ea' or 'ip'; precision 'fp64' or 'bf16x3'.
    """

    def __init__(self, eps, B, nocc, order=3, kind="ea", precision="fp64", max_space_per_root=8, max_iter=100,
                 nguess_extra=2, res_tol=0.0, aux_chunk=0, keep_per_root=2, contractions=-1, refine=1,
                 transition_order=0, refine_res_tol=0.0, m11_on_the_fly=0, tune_cache=None, cuda_graphs=0, lean=-1):
        lib = load_library()
        self._lib = lib
        opt = Options()
        lib.adc_default_options(ctypes.byref(opt))
        opt.precision = PRECISIONS[precision]
        opt.max_space_per_root = max_space_per_root
        opt.max_iter = max_iter
        opt.nguess_extra = nguess_extra
        opt.res_tol = res_tol
        opt.aux_chunk = aux_chunk
        opt.keep_per_root = keep_per_root
        opt.contractions = contractions
        opt.refine = refine
        opt.transition_order = transition_order
        opt.refine_res_tol = refine_res_tol
        opt.m11_on_the_fly = m11_on_the_fly
        opt.tune_cache = None if tune_cache is None else os.fsencode(tune_cache)
        opt.cuda_graphs = cuda_graphs
        opt.lean = lean
        self._solver = dict(max_space_per_root=max_space_per_root, max_iter=max_iter, nguess_extra=nguess_extra,
                            res_tol=res_tol, keep_per_root=keep_per_root, refine=refine,
                            transition_order=transition_order, refine_res_tol=refine_res_tol,
                            cuda_graphs=cuda_graphs)
        if isinstance(eps, np.ndarray):
            eps = np.ascontiguousarray(eps, dtype=np.float64)
            B = np.ascontiguousarray(B, dtype=np.float64)
        else:
            eps = eps.contiguous().double()
            B = B.contiguous().double()
        naux, nmo = B.shape[0], B.shape[1]
        self.nocc, self.nvir, self.naux, self.order, self.kind = nocc, nmo - nocc, naux, order, kind
        pe, dev = _ptr(eps)
        pb, _ = _ptr(B)
        h = ctypes.c_void_p()
        rc = lib.adc_setup(pe, pb, nocc, nmo - nocc, naux, order, ADC_EA if kind == "ea" else ADC_IP,
                           ctypes.byref(opt), dev, ctypes.byref(h))
        if rc != ADC_OK:
            raise ADCError(rc, lib.adc_last_error(None).decode())
        self._h = h
        d = ctypes.c_longlong()
        lib.adc_dim(h, ctypes.byref(d))
        self.dim = d.value

    def _check(self, rc):
        if rc != ADC_OK:
            raise ADCError(rc, self._lib.adc_last_error(self._h).decode())

    def set_stream(self, stream_ptr: int):
        self._check(self._lib.adc_set_stream(self._h, ctypes.c_void_p(stream_ptr)))

    def sigma(self, X, out=None):
        """sigma = M X for X [nvec, dim] (numpy -> numpy, CUDA tensor -> CUDA tensor)."""
        if isinstance(X, np.ndarray):
            X = np.ascontiguousarray(np.atleast_2d(X), dtype=np.float64)
            S = np.empty_like(X) if out is None else out
        else:
            X = X.contiguous()
            if X.dim() == 1:
                X = X.unsqueeze(0)
            S = X.new_empty(X.shape) if out is None else out
        assert X.shape[-1] == self.dim
        px, dev = _ptr(X)
        ps, _ = _ptr(S)
        self._check(self._lib.adc_sigma(self._h, px, ps, X.shape[0], dev))
        return S

    def davidson(self, nroots, tol=1e-8, guess=None, want_vectors=False):
        """(energies, spectroscopic factors, vectors or None, stats dict)."""
        e = np.zeros(nroots)
        p = np.zeros(nroots)
        vec = np.zeros((nroots, self.dim)) if want_vectors else None
        st = np.zeros(8)
        g = None if guess is None else np.ascontiguousarray(guess, dtype=np.float64)
        rc = self._lib.adc_davidson(self._h, nroots, tol, None if g is None else g.ctypes.data, e.ctypes.data,
                                    p.ctypes.data, None if vec is None else vec.ctypes.data, st.ctypes.data)
        stats = dict(iterations=int(st[0]), sigma_vectors=int(st[1]), seconds=st[2], max_residual=st[3],
                     sigma_seconds=st[4], refine_shift=st[5], refine_seconds=st[6], mlp_fallbacks=int(st[7]), status=rc)
        if rc not in (ADC_OK, ADC_ERR_NOT_CONVERGED):
            self._check(rc)
        return e, p, vec, stats

    def set_options(self, **kw):
        """Change solver options (max_space_per_root, max_iter, nguess_extra, res_tol, keep_per_root, refine,
        transition_order, refine_res_tol)."""
        opt = Options()
        self._lib.adc_default_options(ctypes.byref(opt))
        for k in ("max_space_per_root", "max_iter", "nguess_extra", "res_tol", "keep_per_root", "refine",
                  "transition_order", "refine_res_tol", "cuda_graphs"):
            setattr(opt, k, kw.pop(k, self._solver[k]))
        if kw:
            raise TypeError(f"not a solver option: {sorted(kw)}")
        self._check(self._lib.adc_set_options(self._h, ctypes.byref(opt)))
        self._solver = {k: getattr(opt, k) for k in self._solver}

    def set_mlp(self, weights):
        """Use the learned preconditioner with these weights (None: the diagonal one)."""
        if weights is None:
            self._check(self._lib.adc_set_mlp(self._h, None))
        else:
            w = np.ascontiguousarray(weights, dtype=np.float32)
            self._check(self._lib.adc_set_mlp(self._h, w.ctypes.data))

    def mlp_samples(self, nroots, iters=(1, 2, 3, 4, 6, 8, 10, 14), per_vector=100_000, seed=0, exact_tol=1e-10):
        """(d, blk, r, t) training samples of the learned preconditioner (adc_mlp_samples)."""
        it = np.ascontiguousarray(iters, dtype=np.int32)
        n = self._lib.adc_mlp_nsamples(self._h, nroots, it.size, per_vector)
        if n < 0:
            raise ADCError(ADC_ERR_ARG, "adc_mlp_nsamples: invalid argument")
        d, r, t = np.zeros(n), np.zeros(n), np.zeros(n)
        blk = np.zeros(n, dtype=np.uint8)
        self._check(self._lib.adc_mlp_samples(self._h, nroots, it.ctypes.data, it.size, per_vector, seed, exact_tol,
                                              d.ctypes.data, blk.ctypes.data, r.ctypes.data, t.ctypes.data, n))
        return d, blk, r, t

    def mp_energy(self):
        """MP correlation energies (E(2),) for ADC(2) or (E(2), E(3)) for ADC(3), Eh."""
        e = np.zeros(2)
        self._check(self._lib.adc_mp_energy(self._h, e.ctypes.data, 2))
        return tuple(float(x) for x in e[: self.order - 1])

    def get(self, name, shape):
        out = np.zeros(int(np.prod(shape)))
        self._check(self._lib.adc_get_tensor(self._h, name.encode(), out.ctypes.data, out.size))
        return out.reshape(shape)

    def kernel_timing(self, enable: bool):
        """Start (True) or stop (False) live timing of the tensor-core launches.

        On stop returns dict(launches, ms, algo_flops, mma_flops, kernels) over all tensor-core GEMM
        launches, and the same for the DF-ladder GEMMs alone (ladder_launches, ladder_ms, ...)."""
        out = np.zeros(9)
        self._check(self._lib.adc_kernel_timing(self._h, 1 if enable else 0, out.ctypes.data))
        if enable:
            return None
        return dict(launches=int(out[0]), ms=out[1], algo_flops=out[2], mma_flops=out[3], kernels=int(out[4]),
                    ladder_launches=int(out[5]), ladder_ms=out[6], ladder_algo_flops=out[7], ladder_mma_flops=out[8])

    def kernel_launches(self):
        """The launches of the last kernel_timing bracket: array [n, 7] of M, N, K, tile width,
        algorithmic flops, milliseconds, ladder (1) or other contraction (0)."""
        n = self._lib.adc_kernel_launches(self._h, None, 0)
        if n < 0:
            self._check(int(n))
        out = np.zeros((max(n, 1), 7))
        r = self._lib.adc_kernel_launches(self._h, out.ctypes.data, out.size)
        if r < 0:
            self._check(int(r))
        return out[:n]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.adc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ADCBatch:
    """Many independent closed-shell systems, set up and solved concurrently
    (adc_setup_batch / adc_davidson_batch): each system on its own CUDA stream
    and host thread.  systems: list of (eps, B, nocc) float64 numpy arrays."""

    def __init__(self, systems, order=3, kind="ip", precision="bf16x3", **opts):
        lib = load_library()
        self._lib = lib
        opt = Options()
        lib.adc_default_options(ctypes.byref(opt))
        opt.precision = PRECISIONS[precision]
        for k, val in opts.items():
            if not hasattr(opt, k):
                raise TypeError(f"unknown option {k}")
            setattr(opt, k, val)
        self._keep = []
        n = len(systems)
        eps_p = (ctypes.c_void_p * n)()
        b_p = (ctypes.c_void_p * n)()
        no, nv, nq = (ctypes.c_int * n)(), (ctypes.c_int * n)(), (ctypes.c_int * n)()
        for i, (eps, B, nocc) in enumerate(systems):
            eps = np.ascontiguousarray(eps, dtype=np.float64)
            B = np.ascontiguousarray(B, dtype=np.float64)
            self._keep += [eps, B]
            eps_p[i], b_p[i] = eps.ctypes.data, B.ctypes.data
            no[i], nv[i], nq[i] = nocc, B.shape[1] - nocc, B.shape[0]
        handles = (ctypes.c_void_p * n)()
        rc = lib.adc_setup_batch(n, ctypes.cast(eps_p, ctypes.c_void_p), ctypes.cast(b_p, ctypes.c_void_p),
                                 ctypes.cast(no, ctypes.c_void_p), ctypes.cast(nv, ctypes.c_void_p),
                                 ctypes.cast(nq, ctypes.c_void_p), order, ADC_EA if kind == "ea" else ADC_IP,
                                 ctypes.byref(opt), 0, ctypes.cast(handles, ctypes.c_void_p))
        self._keep = []
        if rc != ADC_OK:
            raise ADCError(rc, lib.adc_last_error(None).decode())
        self._h = handles
        self.n = n

    def davidson(self, nroots, tol=1e-6):
        """(energies [n, nroots], spectroscopic factors [n, nroots], stats [n, 8], status [n])."""
        e = np.zeros((self.n, nroots))
        p = np.zeros((self.n, nroots))
        st = np.zeros((self.n, 8))
        status = (ctypes.c_int * self.n)()
        rc = self._lib.adc_davidson_batch(ctypes.cast(self._h, ctypes.c_void_p), self.n, nroots, tol, e.ctypes.data,
                                          p.ctypes.data, st.ctypes.data, ctypes.cast(status, ctypes.c_void_p))
        status = np.array(list(status))
        if rc not in (ADC_OK, ADC_ERR_NOT_CONVERGED):
            bad = int(np.nonzero(status != ADC_OK)[0][0])
            raise ADCError(rc, self._lib.adc_last_error(self._h[bad]).decode())
        return e, p, st, status

    def close(self):
        if getattr(self, "_h", None) is not None:
            for i in range(self.n):
                self._lib.adc_destroy(self._h[i])
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_nweights():
    return load_library().adc_mlp_nweights()


def _mlp_samples(d, blk, r, t):
    d = np.ascontiguousarray(d, dtype=np.float64)
    blk = np.ascontiguousarray(blk, dtype=np.uint8)
    r = np.ascontiguousarray(r, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    if not (d.shape == blk.shape == r.shape == t.shape) or d.ndim != 1:
        raise ValueError("samples must be 1-D arrays of one length")
    return d, blk, r, t


def mlp_loss_grad(weights, d, blk, r, t):
    """(loss, gradient) of the learned preconditioner on samples (adc_mlp_loss_grad)."""
    lib = load_library()
    w = np.ascontiguousarray(weights, dtype=np.float32)
    d, blk, r, t = _mlp_samples(d, blk, r, t)
    grad = np.zeros(lib.adc_mlp_nweights(), dtype=np.float32)
    loss = ctypes.c_double()
    rc = lib.adc_mlp_loss_grad(w.ctypes.data, d.ctypes.data, blk.ctypes.data, r.ctypes.data, t.ctypes.data, d.size,
                               grad.ctypes.data, ctypes.byref(loss))
    if rc != ADC_OK:
        raise ADCError(rc, lib.adc_last_error(None).decode())
    return loss.value, grad


def mlp_train(weights, d, blk, r, t, steps=500, lr=1e-3):
    """Full-batch Adam on the GPU (adc_mlp_train); returns (weights, loss history)."""
    lib = load_library()
    w = np.array(weights, dtype=np.float32)
    d, blk, r, t = _mlp_samples(d, blk, r, t)
    hist = np.zeros(max(steps, 1))
    rc = lib.adc_mlp_train(w.ctypes.data, d.ctypes.data, blk.ctypes.data, r.ctypes.data, t.ctypes.data, d.size, steps,
                           float(lr), hist.ctypes.data)
    if rc != ADC_OK:
        raise ADCError(rc, lib.adc_last_error(None).decode())
    return w, hist[:steps]


class ADCUnrestricted:
    """Unrestricted (open-shell) reference for EA/IP-UADC(n) sigma products (FP64).

    eps_a, eps_b [nmo] and B_a, B_b [naux, nmo, nmo] are float64 numpy arrays
    (alpha / beta orbitals, occupied first).  The vector layout is the one of
    adc_setup_unrestricted: spin orbitals ordered occupied alpha, occupied
    beta, virtual alpha, virtual beta; EA [1p | (i, a<b)], IP [1h | (i<j, a)].
    """

    def __init__(self, eps_a, eps_b, B_a, B_b, nocc_a, nocc_b, order=3, kind="ea", aux_chunk=0, precision="fp64",
                 refine=1, refine_res_tol=0.0):
        lib = load_library()
        self._lib = lib
        arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (eps_a, eps_b, B_a, B_b)]
        naux, nmo = arrs[2].shape[0], arrs[2].shape[1]
        self.order, self.kind = order, kind
        opt = Options()
        lib.adc_default_options(ctypes.byref(opt))
        opt.precision, opt.aux_chunk, opt.refine, opt.refine_res_tol = PRECISIONS[precision], aux_chunk, refine, refine_res_tol
        self._solver = dict(refine=refine, refine_res_tol=refine_res_tol)
        h = ctypes.c_void_p()
        rc = lib.adc_setup_unrestricted(*[a.ctypes.data for a in arrs], nocc_a, nocc_b, nmo, naux, order,
                                        ADC_EA if kind == "ea" else ADC_IP, ctypes.byref(opt), ctypes.byref(h))
        if rc != ADC_OK:
            raise ADCError(rc, lib.adc_last_error(None).decode())
        self._h = h
        d = ctypes.c_longlong()
        lib.adc_dim(h, ctypes.byref(d))
        self.dim = d.value

    def _check(self, rc):
        if rc != ADC_OK:
            raise ADCError(rc, self._lib.adc_last_error(self._h).decode())

    def davidson(self, nroots, tol=1e-8, want_vectors=False, res_tol=0.0, max_iter=100, max_space_per_root=8):
        """(energies, spectroscopic factors (one spin-orbital component), vectors or None, stats dict)."""
        opt = Options()
        self._lib.adc_default_options(ctypes.byref(opt))
        opt.res_tol, opt.max_iter, opt.max_space_per_root = res_tol, max_iter, max_space_per_root
        opt.refine, opt.refine_res_tol = self._solver["refine"], self._solver["refine_res_tol"]
        self._check(self._lib.adc_set_options(self._h, ctypes.byref(opt)))
        e = np.zeros(nroots)
        p = np.zeros(nroots)
        vec = np.zeros((nroots, self.dim)) if want_vectors else None
        st = np.zeros(8)
        rc = self._lib.adc_davidson(self._h, nroots, tol, None, e.ctypes.data, p.ctypes.data,
                                    None if vec is None else vec.ctypes.data, st.ctypes.data)
        stats = dict(iterations=int(st[0]), sigma_vectors=int(st[1]), seconds=st[2], max_residual=st[3], status=rc)
        if rc not in (ADC_OK, ADC_ERR_NOT_CONVERGED):
            self._check(rc)
        return e, p, vec, stats

    def sigma(self, X):
        """sigma = M X (EA) or -M_- X (IP) for host X [nvec, dim]."""
        X = np.ascontiguousarray(np.atleast_2d(X), dtype=np.float64)
        assert X.shape[-1] == self.dim
        S = np.empty_like(X)
        self._check(self._lib.adc_sigma(self._h, X.ctypes.data, S.ctypes.data, X.shape[0], 0))
        return S

    def get(self, name, shape):
        out = np.zeros(int(np.prod(shape)))
        self._check(self._lib.adc_get_tensor(self._h, name.encode(), out.ctypes.data, out.size))
        return out.reshape(shape)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.adc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
