"""The 1p-1p / 1h-1h block applied on the fly (m11_on_the_fly = 1; the paper's
alternative to precomputing the block in step 3, Sec. III A) against the
tier-2 oracle: sigma element by element in FP64 (1e-11 relative, the
rounding-order bound of the FP64 path) and in mixed precision (the split-BF16
bound of the mixed tests, 3e-5 of max |sigma|), EA and IP, ADC(2) and ADC(3),
with ragged sizes; and roots through the Davidson solver, whose preconditioner
then takes the zeroth-order one-particle energies, against dense
diagonalisation."""
import numpy as np
import pytest

from adc_inputs import make_system
from oracle.spinadapted import SpinAdaptedADC

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(4, 14, 40, 0), (5, 37, 61, 3)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"o{c[0]}v{c[1]}Q{c[2]}")
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_sigma_on_the_fly_fp64(kind, order, case):
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = case
    s = make_system(o, v, naux, seed=seed)
    ref = SpinAdaptedADC(s.eps, o, s.B, order, kind)
    g = ADC(s.eps, s.B, o, order=order, kind=kind, precision="fp64", m11_on_the_fly=1)
    X = np.random.default_rng(7).standard_normal((3, g.dim))
    Sg = g.sigma(X)
    Sr = ref.sigma(X)
    g.close()
    assert np.abs(Sg - Sr).max() <= 1e-11 * np.abs(Sr).max(), np.abs(Sg - Sr).max()


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_sigma_on_the_fly_mixed(kind):
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = 6, 70, 150, 1
    s = make_system(o, v, naux, seed=seed)
    ref = SpinAdaptedADC(s.eps, o, s.B, 3, kind)
    g = ADC(s.eps, s.B, o, order=3, kind=kind, precision="bf16x3", m11_on_the_fly=1)
    X = np.random.default_rng(9).standard_normal((3, g.dim))
    Sg = g.sigma(X)
    Sr = ref.sigma(X)
    g.close()
    assert np.abs(Sg - Sr).max() <= 3e-5 * np.abs(Sr).max(), np.abs(Sg - Sr).max()


@pytest.mark.parametrize("kind", ["ea", "ip"])
def test_roots_on_the_fly(kind):
    from oracle.davidson import dense_roots
    from paper_2012_06714_gb300 import ADC

    o, v, naux = 4, 14, 40
    s = make_system(o, v, naux, seed=0)
    ref = SpinAdaptedADC(s.eps, o, s.B, 3, kind)
    w, _ = dense_roots(ref, 3)
    g = ADC(s.eps, s.B, o, order=3, kind=kind, precision="fp64", m11_on_the_fly=1, res_tol=1e-6)
    e, p, _, st = g.davidson(3, tol=1e-10)
    g.close()
    assert st["status"] == 0
    assert np.abs(e - w).max() < 1e-8, np.abs(e - w).max()
