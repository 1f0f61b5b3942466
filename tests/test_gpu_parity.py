"""GPU path (C ABI) against the CPU oracle, element by element.

FP64 path: sigma, setup intermediates and roots equal the spin-adapted oracle
to rounding (relative 1e-11 on sigma).  Sizes span several GEMM tiles with
ragged tails (nvir not a multiple of 8/64, nocc odd)."""
import numpy as np
import pytest

from adc_inputs import make_system
from oracle.davidson import davidson as oracle_davidson
from oracle.davidson import dense_roots, spectroscopic_factors
from oracle.spinadapted import SpinAdaptedADC

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(3, 13, 24, 0), (5, 20, 80, 0), (7, 37, 61, 3)]


@pytest.fixture(scope="module")
def lib():
    from paper_2012_06714_gb300 import load_library

    return load_library()


def _mk(o, v, naux, seed):
    return make_system(o, v, naux, seed=seed)


@pytest.mark.parametrize("kind", ["ea", "ip"])
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"o{c[0]}v{c[1]}Q{c[2]}")
def test_sigma_fp64(lib, kind, order, case):
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = case
    s = _mk(o, v, naux, seed)
    gpu = ADC(s.eps, s.B, o, order=order, kind=kind)
    ref = SpinAdaptedADC(s.eps, o, s.B, order, kind)
    assert gpu.dim == ref.dim
    X = np.random.default_rng(7).standard_normal((4, gpu.dim))
    Sg = gpu.sigma(X)
    Sr = ref.sigma(X)
    assert np.abs(Sg - Sr).max() <= 1e-11 * np.abs(Sr).max()
    # device pointers give the same result
    Sd = gpu.sigma(torch.from_numpy(X).cuda()).cpu().numpy()
    assert np.abs(Sd - Sg).max() <= 1e-13 * np.abs(Sr).max()
    gpu.close()


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_setup_intermediates(lib, kind):
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = CASES[2]
    s = _mk(o, v, naux, seed)
    gpu = ADC(s.eps, s.B, o, order=3, kind=kind)
    ref = SpinAdaptedADC(s.eps, o, s.B, 3, kind)
    n1 = ref.n1
    assert np.abs(gpu.get("M11", (n1, n1)) - ref.M11).max() < 1e-12
    assert np.abs(gpu.get("t2", (o, o, v, v)) - ref.t).max() < 1e-13
    assert np.abs(gpu.get("t2_2", (o, o, v, v)) - ref.t_2).max() < 1e-13
    assert np.abs(gpu.get("t1_2", (o, v)) - ref.t1_2).max() < 1e-13
    assert np.abs(gpu.get("t1_3", (o, v)) - ref.t1_3).max() < 1e-13
    e_ref = ref.mp_energies()
    assert np.abs(np.array(gpu.mp_energy()) - e_ref).max() < 1e-12 * abs(e_ref[0])
    assert np.abs(gpu.get("diag", (ref.dim,)) - ref.diagonal()).max() < 1e-12
    gpu.close()


@pytest.fixture(scope="module")
def chunked_case():
    o, v, naux = 11, 97, 1500
    s = _mk(o, v, naux, 5)
    return s, SpinAdaptedADC(s.eps, o, s.B, 3, "ip")


@pytest.mark.parametrize("precision", ["fp64", "bf16x3"])
def test_third_order_singles_auxiliary_chunks(lib, chunked_case, precision):
    """t_i^a(3) with the auxiliary index split into two chunks (1500 = 1039 + 461
    at nocc 11, nvir 97, chunk set through aux_chunk) against the oracle, and in
    one chunk (the automatic size); the mixed path forms it in the setup's
    FP32-accurate contractions (relative 1e-6 of the largest element)."""
    from paper_2012_06714_gb300 import ADC

    s, ref = chunked_case
    o, v = 11, 97
    one = ADC(s.eps, s.B, o, order=3, kind="ip", precision=precision)
    whole = one.get("t1_3", (o, v))
    one.close()
    gpu = ADC(s.eps, s.B, o, order=3, kind="ip", precision=precision, aux_chunk=1039)
    got = gpu.get("t1_3", (o, v))
    gpu.close()
    scale = np.abs(ref.t1_3).max()
    assert scale > 1e-4
    assert np.abs(got - ref.t1_3).max() <= (1e-12 if precision == "fp64" else 1e-6) * scale
    assert np.abs(whole - ref.t1_3).max() <= (1e-12 if precision == "fp64" else 1e-6) * scale


@pytest.mark.parametrize("kind", ["ea", "ip"])
@pytest.mark.parametrize("order", [2, 3])
def test_davidson_fp64_small(lib, kind, order):
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = 5, 20, 80, 0
    s = _mk(o, v, naux, seed)
    gpu = ADC(s.eps, s.B, o, order=order, kind=kind, res_tol=1e-9)
    ref = SpinAdaptedADC(s.eps, o, s.B, order, kind)
    w, Y = dense_roots(ref, 4)
    e, p, vec, st = gpu.davidson(4, tol=1e-10, want_vectors=True)
    assert st["status"] == 0
    assert np.abs(e - w).max() < 1e-8
    pr = spectroscopic_factors(ref, vec)
    assert np.abs(p - pr).max() < 1e-10
    assert np.abs(p - spectroscopic_factors(ref, Y)).max() < 1e-7
    if order == 3:
        # second-order transition moments on request (transition_order = 2)
        gpu.set_options(transition_order=2)
        e2, p2, vec2, _ = gpu.davidson(4, tol=1e-10, want_vectors=True)
        assert np.abs(p2 - spectroscopic_factors(ref, vec2, 2)).max() < 1e-10
        assert np.abs(p2 - p).max() > 1e-6
    gpu.close()


def test_invalid_arguments(lib):
    from paper_2012_06714_gb300 import ADC
    from paper_2012_06714_gb300._lib import ADCError

    s = _mk(2, 5, 8, 0)
    gpu = ADC(s.eps, s.B, 2, order=2, kind="ea")
    with pytest.raises(ADCError):
        gpu.davidson(0)
    with pytest.raises(ADCError):
        gpu.davidson(gpu.dim + 1)
    gpu.close()


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_spectroscopic_amplitudes_and_spectrum(kind):
    """X from adc_get_tensor("X") reproduces the returned factors (P = 2 sum_p X^2,
    Appendix) and the propagator route of the spectral function (Eqs. g_adc,
    spec_function) equals adc_spectrum's P route."""
    from oracle.spectrum import spectral_function
    from paper_2012_06714_gb300 import ADC, spectrum

    o, v, naux = 4, 14, 40
    s = make_system(o, v, naux, seed=3)
    g = ADC(s.eps, s.B, o, order=3, kind=kind, precision="fp64")
    e, p, _, st = g.davidson(3, tol=1e-10)
    X = g.get("X", (3, o + v))
    g.close()
    assert np.abs(2.0 * (X * X).sum(axis=1) - p).max() < 1e-12
    w = np.linspace(e.min() - 0.2, e.max() + 0.2, 101)
    assert np.abs(spectrum(e, p, w, 0.01) - 2.0 * spectral_function(X.T, e, w, 0.01)).max() < 1e-10
