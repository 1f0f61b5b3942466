"""Mixed-precision (BF16x3 tensor-core ladder) GPU path against the FP64 oracle.

Tolerance: every operand is split x = hi + lo with hi, lo in BF16, so each
operand keeps 16 significant bits (relative representation error <= 2^-17)
and a product loses at most ~3 * 2^-17 relative (the dropped lo*lo term is
2^-16 smaller still); the intermediate Z is split again (another 2^-17) and
FP32 accumulation within one auxiliary chunk adds <= K2 * 2^-24.  Summed over
terms of mixed sign, the ladder error is bounded by ~1e-5 times
sum_Q |B^Q| |X| |B^Q|; the tests use 3e-5 of max |sigma| (the ladder is the
largest term) and the roots are required to agree with FP64 to 1e-6 Eh."""
import numpy as np
import pytest

from adc_inputs import make_system
from oracle.spinadapted import SpinAdaptedADC

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(4, 14, 40, 0), (3, 37, 61, 3), (6, 70, 150, 1)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"o{c[0]}v{c[1]}Q{c[2]}")
def test_sigma_bf16x3_vs_oracle(case):
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = case
    s = make_system(o, v, naux, seed=seed)
    gpu = ADC(s.eps, s.B, o, order=3, kind="ea", precision="bf16x3")
    ref = SpinAdaptedADC(s.eps, o, s.B, 3, "ea")
    X = np.random.default_rng(5).standard_normal((3, gpu.dim))
    Sg = gpu.sigma(X)
    Sr = ref.sigma(X)
    # ladder alone, to state the error relative to the term it comes from
    L = np.abs(ref.ladder(X[:, v:].reshape(3, o, v, v))).max()
    err = np.abs(Sg - Sr).max()
    assert err <= 3e-5 * max(L, np.abs(Sr).max()), (err, L)
    assert np.isfinite(Sg).all()
    gpu.close()


def test_setup_bf16x3_amplitudes():
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = CASES[1]
    s = make_system(o, v, naux, seed=seed)
    gpu = ADC(s.eps, s.B, o, order=3, kind="ea", precision="bf16x3")
    ref = SpinAdaptedADC(s.eps, o, s.B, 3, "ea")
    t2 = gpu.get("t2_2", (o, o, v, v))
    assert np.abs(t2 - ref.t_2).max() <= 3e-5 * np.abs(ref.t_2).max()
    M = gpu.get("M11", (v, v))
    assert np.abs(M - ref.M11).max() <= 1e-6
    gpu.close()


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_roots_bf16x3_vs_fp64(kind):
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = 6, 40, 100, 2
    s = make_system(o, v, naux, seed=seed)
    g64 = ADC(s.eps, s.B, o, order=3, kind=kind, precision="fp64", res_tol=1e-6)
    gmx = ADC(s.eps, s.B, o, order=3, kind=kind, precision="bf16x3", res_tol=1e-6)
    e64, p64, _, _ = g64.davidson(4, tol=1e-9)
    emx, pmx, _, st = gmx.davidson(4, tol=1e-9)
    assert st["status"] == 0
    assert np.abs(e64 - emx).max() < 1e-6
    assert np.abs(p64 - pmx).max() < 1e-4
    g64.close()
    gmx.close()
