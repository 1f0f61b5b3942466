"""Mixed-precision (tensor-core BF16 split ladder) GPU path against the FP64 oracle.

Tolerance: every operand is split x = hi + lo with hi, lo in BF16, so each
operand keeps 16 significant bits (relative representation error <= 2^-17)
and a product loses at most ~3 * 2^-17 relative (the dropped lo*lo term is
2^-16 smaller still); the intermediate Z is split again (another 2^-17).  The
tensor core's FP32 accumulation truncates (about a quarter ulp, 2^-26
relative, per MMA, always toward zero); the kernel adds its tensor-memory
partial sums into round-to-nearest FP32 registers every 16 K blocks (192
MMAs, <= ~3e-6 relative drift) in sigma and every K block in the setup
ladder and the final refinement.  Summed over terms of mixed sign, the sigma
ladder error is bounded by ~1e-5 times sum_Q |B^Q| |X| |B^Q|; the tests use
3e-5 of max |sigma| (the ladder is the largest term).  t2(2) and M_11 carry
errors of ~1e-6 relative, and the refined roots agree with FP64 to 5e-7 Eh."""
import numpy as np
import pytest

from adc_inputs import make_system
from oracle.spinadapted import SpinAdaptedADC

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(4, 14, 40, 0), (3, 37, 61, 3), (6, 70, 150, 1)]
TOL = {"bf16x3": 3e-5}
TOL_SETUP = 3e-6
TOL_E = {"bf16x3": 5e-7}


@pytest.mark.parametrize("prec", ["bf16x3"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"o{c[0]}v{c[1]}Q{c[2]}")
def test_sigma_mixed_vs_oracle(case, prec):
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = case
    s = make_system(o, v, naux, seed=seed)
    gpu = ADC(s.eps, s.B, o, order=3, kind="ea", precision=prec)
    ref = SpinAdaptedADC(s.eps, o, s.B, 3, "ea")
    X = np.random.default_rng(5).standard_normal((3, gpu.dim))
    Sg = gpu.sigma(X)
    Sr = ref.sigma(X)
    # ladder alone, to state the error relative to the term it comes from
    L = np.abs(ref.ladder(X[:, v:].reshape(3, o, v, v))).max()
    err = np.abs(Sg - Sr).max()
    assert err <= TOL[prec] * max(L, np.abs(Sr).max()), (err, L)
    assert np.isfinite(Sg).all()
    gpu.close()


@pytest.mark.parametrize("prec", ["bf16x3"])
def test_setup_mixed_amplitudes(prec):
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = CASES[1]
    s = make_system(o, v, naux, seed=seed)
    gpu = ADC(s.eps, s.B, o, order=3, kind="ea", precision=prec)
    ref = SpinAdaptedADC(s.eps, o, s.B, 3, "ea")
    t2 = gpu.get("t2_2", (o, o, v, v))
    assert np.abs(t2 - ref.t_2).max() <= TOL_SETUP * np.abs(ref.t_2).max()
    M = gpu.get("M11", (v, v))
    assert np.abs(M - ref.M11).max() <= 2e-7
    gpu.close()


@pytest.mark.parametrize("prec", ["bf16x3"])
@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_roots_mixed_vs_fp64(kind, prec):
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = 6, 40, 100, 2
    s = make_system(o, v, naux, seed=seed)
    g64 = ADC(s.eps, s.B, o, order=3, kind=kind, precision="fp64", res_tol=1e-7)
    gmx = ADC(s.eps, s.B, o, order=3, kind=kind, precision=prec, res_tol=1e-5, refine_res_tol=1e-7)
    e64, p64, _, _ = g64.davidson(4, tol=1e-9)
    emx, pmx, _, st = gmx.davidson(4, tol=1e-9)
    assert st["status"] == 0
    assert np.abs(e64 - emx).max() < TOL_E[prec], np.abs(e64 - emx).max()
    # vectors converged under the accurate operator: P within the target of 1e-6
    assert np.abs(p64 - pmx).max() < 1e-6, np.abs(p64 - pmx).max()
    g64.close()
    gmx.close()


def test_refinement_moves_roots_toward_fp64():
    """The final refinement (accurate ladder on the converged roots, other
    contractions FP32-accurate or FP64) changes the energies and lands within
    TOL_E of FP64."""
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = 8, 60, 160, 4
    s = make_system(o, v, naux, seed=seed)
    g64 = ADC(s.eps, s.B, o, order=3, kind="ea", precision="fp64", res_tol=1e-6)
    e64, p64, _, _ = g64.davidson(3, tol=1e-9)
    g64.close()
    res = {}
    for rf in (0, 1, 2):
        g = ADC(s.eps, s.B, o, order=3, kind="ea", precision="bf16x3", res_tol=1e-6, refine=rf)
        e, p, vec, st = g.davidson(3, tol=1e-9, want_vectors=True)
        assert st["status"] == 0
        res[rf] = (e, p, st)
        g.close()
    e0, _, st0 = res[0]
    assert st0["refine_shift"] == 0.0 and st0["refine_seconds"] == 0.0
    assert np.abs(e0 - e64).max() < 2e-6
    for rf in (1, 2):  # other contractions FP32-accurate (1) or FP64 (2)
        e1, p1, st1 = res[rf]
        assert st1["refine_shift"] > 0.0
        assert np.abs(e1 - e64).max() < TOL_E["bf16x3"], (rf, np.abs(e1 - e64).max())
        assert np.abs(p1 - p64).max() < 1e-4


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_tensor_core_contractions_vs_fp32(kind):
    """sigma with the large non-ladder contractions on the tensor-core split-BF16
    GEMM (contractions=2, the mixed default) against the same sigma with
    FP32-accurate contractions (contractions=1, checked against the oracle
    above); the system is large enough for those contractions to take the
    tensor-core path.  Bound: the split-BF16 error (~1e-5 of each term's
    magnitude), 3e-5 of max |sigma|."""
    from paper_2012_06714_gb300 import ADC

    o, v, naux = (24, 256, 300) if kind == "ea" else (48, 160, 300)
    s = make_system(o, v, naux, seed=6)
    g2 = ADC(s.eps, s.B, o, order=3, kind=kind, precision="bf16x3", contractions=2)
    g1 = ADC(s.eps, s.B, o, order=3, kind=kind, precision="bf16x3", contractions=1)
    X = np.random.default_rng(8).standard_normal((4, g2.dim))
    S2 = g2.sigma(X)
    S1 = g1.sigma(X)
    err = np.abs(S2 - S1).max()
    assert err <= 3e-5 * np.abs(S1).max(), (err, np.abs(S1).max())
    g1.close()
    g2.close()
