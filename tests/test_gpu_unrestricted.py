"""GPU EA/IP-UADC(n) sigma (unrestricted open-shell references, FP64) against
the density-fitted unrestricted oracle, element by element: amplitudes, the
one-particle block and sigma = M Y on random vectors, for nocc_a != nocc_b and
a case with ragged sizes."""
import numpy as np
import pytest

from adc_inputs import make_open_shell_system

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(3, 2, 7, 20, 5, 2.0), (5, 4, 23, 41, 2, 1.0)]  # nocc_a, nocc_b, nmo, naux, seed, B scale


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"a{c[0]}b{c[1]}n{c[2]}")
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_unrestricted_sigma_fp64(kind, order, case):
    from oracle.unrestricted import UnrestrictedDFADC
    from paper_2012_06714_gb300 import ADCUnrestricted

    na, nb, nmo, naux, seed, scale = case
    s = make_open_shell_system(na, nb, nmo, naux, seed=seed)
    s.B_a *= scale
    s.B_b *= scale
    ref = UnrestrictedDFADC(s, order, kind)
    gpu = ADCUnrestricted(s.eps_a, s.eps_b, s.B_a, s.B_b, na, nb, order=order, kind=kind)
    assert gpu.dim == ref.dim
    o, v = ref.no, ref.nv
    assert np.abs(gpu.get("t2", (o, o, v, v)) - ref.t2_1).max() < 1e-13
    if order == 3:
        assert np.abs(gpu.get("t2_2", (o, o, v, v)) - ref.t2_2).max() < 1e-13
        assert np.abs(gpu.get("t1_2", (o, v)) - ref.t1_2).max() < 1e-13
    n1 = ref.n1
    assert np.abs(gpu.get("M11", (n1, n1)) - ref.M11).max() < 1e-12
    X = np.random.default_rng(3).standard_normal((3, gpu.dim))
    Sg = gpu.sigma(X)
    Sr = ref.sigma(X)
    gpu.close()
    assert np.abs(Sg - Sr).max() <= 1e-11 * np.abs(Sr).max()


def test_unrestricted_ip3_coupling_in_auxiliary_chunks():
    """The IP-UADC(3) coupling intermediate sum_e B^Q_ie t_jk^de (naux x o^3 x v)
    is built in auxiliary chunks; 3 functions per chunk (14 chunks, the last
    ragged) give the same sigma as the oracle."""
    from oracle.unrestricted import UnrestrictedDFADC
    from paper_2012_06714_gb300 import ADCUnrestricted

    na, nb, nmo, naux = 5, 4, 23, 41
    s = make_open_shell_system(na, nb, nmo, naux, seed=2)
    ref = UnrestrictedDFADC(s, 3, "ip")
    gpu = ADCUnrestricted(s.eps_a, s.eps_b, s.B_a, s.B_b, na, nb, order=3, kind="ip", aux_chunk=3)
    X = np.random.default_rng(4).standard_normal((2, gpu.dim))
    Sg = gpu.sigma(X)
    Sr = ref.sigma(X)
    gpu.close()
    assert np.abs(Sg - Sr).max() <= 1e-11 * np.abs(Sr).max()


def _group_sums(w, p, tol=1e-6):
    """spectroscopic factors summed over groups of degenerate roots (the vectors of a
    degenerate group are fixed only up to a rotation within it)"""
    out, k = [], 0
    while k < len(w):
        j = k + 1
        while j < len(w) and w[j] - w[j - 1] < tol:
            j += 1
        out.append(p[k:j].sum())
        k = j
    return np.array(out)


@pytest.mark.parametrize("case", [CASES[0], (4, 3, 11, 30, 2, 1.0)], ids=lambda c: f"a{c[0]}b{c[1]}n{c[2]}")
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_unrestricted_roots_and_factors(kind, order, case):
    """UADC Davidson (S = 1) against dense diagonalisation of the oracle's matrix: the
    lowest roots to 1e-8 Eh and their spectroscopic factors (T through order n,
    third-order singles included for ADC(3)) to 1e-6."""
    from oracle.unrestricted import UnrestrictedDFADC
    from paper_2012_06714_gb300 import ADCUnrestricted

    na, nb, nmo, naux, seed, scale = case
    s = make_open_shell_system(na, nb, nmo, naux, seed=seed)
    s.B_a *= scale
    s.B_b *= scale
    ref = UnrestrictedDFADC(s, order, kind)
    w, V = np.linalg.eigh(ref.dense())
    nroots = 3
    if w[nroots] - w[nroots - 1] < 1e-6:  # keep a degenerate group whole
        nroots += 1
    pref = ref.spectroscopic_factors(V[:, :nroots].T)
    gpu = ADCUnrestricted(s.eps_a, s.eps_b, s.B_a, s.B_b, na, nb, order=order, kind=kind)
    if order == 3:
        o, v = ref.no, ref.nv
        assert np.abs(gpu.get("t1_3", (o, v)) - ref.t1_3).max() < 1e-12
    e, p, _, st = gpu.davidson(nroots, tol=1e-10, res_tol=1e-7)
    gpu.close()
    assert st["status"] == 0
    assert np.abs(e - w[:nroots]).max() < 1e-8, (e, w[:nroots])
    assert np.abs(_group_sums(w[:nroots], p) - _group_sums(w[:nroots], pref)).max() < 1e-6, (p, pref)


def test_unrestricted_argument_errors():
    import ctypes

    from paper_2012_06714_gb300 import ADCUnrestricted
    from paper_2012_06714_gb300._lib import ADCError, load_library

    s = make_open_shell_system(1, 0, 2, 4, seed=0)
    with pytest.raises(ADCError):  # one occupied spin orbital: no 2h1p pair
        ADCUnrestricted(s.eps_a, s.eps_b, s.B_a, s.B_b, 1, 0, kind="ip")
    g = ADCUnrestricted(s.eps_a, s.eps_b, s.B_a, s.B_b, 1, 0, order=2, kind="ea")
    L = load_library()
    e = np.zeros(2)
    assert L.adc_davidson(g._h, 0, 1e-6, None, e.ctypes.data, None, None, None) != 0  # nroots < 1
    with pytest.raises(ADCError):  # no beta virtual orbital: no per-spin mixed-precision ladder
        s2 = make_open_shell_system(2, 2, 2, 4, seed=0)
        ADCUnrestricted(s2.eps_a, s2.eps_b, s2.B_a, s2.B_b, 2, 2, order=2, kind="ip", precision="bf16x3")
    assert L.adc_mp_energy(g._h, e.ctypes.data, 2) != 0
    g.close()


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_unrestricted_sigma_mixed(kind):
    """Mixed-precision UADC(3) sigma (the ladder per spin block on the tensor cores with
    split-BF16 operands, the other large contractions on the tensor-core GEMM) against the
    oracle: the split-BF16 bound of the closed-shell mixed tests, 3e-5 of max |sigma|."""
    from oracle.unrestricted import UnrestrictedDFADC
    from paper_2012_06714_gb300 import ADCUnrestricted

    na, nb, nmo, naux = 5, 4, 23, 41
    s = make_open_shell_system(na, nb, nmo, naux, seed=2)
    ref = UnrestrictedDFADC(s, 3, kind)
    gpu = ADCUnrestricted(s.eps_a, s.eps_b, s.B_a, s.B_b, na, nb, order=3, kind=kind, precision="bf16x3")
    X = np.random.default_rng(6).standard_normal((3, gpu.dim))
    Sg = gpu.sigma(X)
    Sr = ref.sigma(X)
    gpu.close()
    assert np.abs(Sg - Sr).max() <= 3e-5 * np.abs(Sr).max(), np.abs(Sg - Sr).max()


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_unrestricted_roots_mixed_vs_fp64(kind):
    """Mixed-precision UADC(3) roots, continued with the accurate operator (FP64 contractions,
    promoted ladder) to residual 1e-7, against the FP64 GPU roots: 1e-6 Eh and P within 1e-6."""
    from paper_2012_06714_gb300 import ADCUnrestricted

    na, nb, nmo, naux = 4, 3, 11, 30
    s = make_open_shell_system(na, nb, nmo, naux, seed=2)
    g64 = ADCUnrestricted(s.eps_a, s.eps_b, s.B_a, s.B_b, na, nb, order=3, kind=kind)
    e64, p64, _, _ = g64.davidson(3, tol=1e-10, res_tol=1e-7)
    g64.close()
    gmx = ADCUnrestricted(s.eps_a, s.eps_b, s.B_a, s.B_b, na, nb, order=3, kind=kind, precision="bf16x3",
                          refine_res_tol=1e-7)
    emx, pmx, _, st = gmx.davidson(3, tol=1e-10, res_tol=1e-5)
    gmx.close()
    assert st["status"] == 0
    assert np.abs(emx - e64).max() < 1e-6, np.abs(emx - e64).max()
    assert np.abs(pmx - p64).max() < 1e-6, np.abs(pmx - p64).max()
