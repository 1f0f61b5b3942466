"""The tile autotuner (adc_options.tune_cache).

A handle with a cache path times each tensor-core problem of its first sigma
once per candidate tile choice (ladder GEMM2 tile width and auxiliary chunk,
generic contraction tile width), keeps the fastest and writes the table.  The
tuned sigma must agree with the oracle within the split-BF16 bound of the
mixed tests (3e-5 of max |sigma|); a second handle reading the same file must
reuse the stored choices -- it writes nothing and its sigma is bitwise equal
to the first handle's."""
import os

import numpy as np
import pytest

from adc_inputs import make_system
from oracle.spinadapted import SpinAdaptedADC

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_tuned_sigma_and_cache_reuse(tmp_path):
    from paper_2012_06714_gb300 import ADC

    o, v, naux = 8, 100, 200
    s = make_system(o, v, naux, seed=5)
    cache = str(tmp_path / "tiles.txt")
    g1 = ADC(s.eps, s.B, o, order=3, kind="ea", precision="bf16x3", tune_cache=cache)
    X = np.random.default_rng(3).standard_normal((4, g1.dim))
    S1 = g1.sigma(X)
    g1.close()
    lines = open(cache).read().split("\n")
    assert any(l.startswith("ladder:") for l in lines) and any(l.startswith("gemm:") for l in lines)
    Sr = SpinAdaptedADC(s.eps, o, s.B, 3, "ea").sigma(X)
    assert np.abs(S1 - Sr).max() <= 3e-5 * np.abs(Sr).max()
    before = os.stat(cache).st_mtime_ns
    g2 = ADC(s.eps, s.B, o, order=3, kind="ea", precision="bf16x3", tune_cache=cache)
    S2 = g2.sigma(X)
    g2.close()
    assert os.stat(cache).st_mtime_ns == before
    assert np.array_equal(S1, S2)
