"""Failure paths of the Davidson solver, made on the host (no GPU fault).

- max_iter = 1: ADC_ERR_NOT_CONVERGED with energies, vectors and statistics
  filled with the best estimates of the first iteration.
- learned-preconditioner weights that are NaN: every learned correction is
  non-finite, each root falls back to the diagonal preconditioner, and the run
  converges to the same roots as the plain diagonal run.
- a NaN element in a caller's guess vector: ADC_ERR_NONFINITE before any work.
- a NaN orbital energy: sigma is non-finite and the solver stops with
  ADC_ERR_NONFINITE instead of returning garbage.
"""
import numpy as np
import pytest

from adc_inputs import make_system

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NOT_CONVERGED, NONFINITE = -4, -6


def _system():
    return make_system(4, 16, 48, seed=2)


def test_max_iter_one_reports_not_converged_with_estimates():
    from paper_2012_06714_gb300 import ADC

    s = _system()
    g = ADC(s.eps, s.B, 4, order=3, kind="ea", precision="fp64", max_iter=1)
    e, p, vec, st = g.davidson(3, tol=1e-9, want_vectors=True)
    g.close()
    assert st["status"] == NOT_CONVERGED
    assert st["iterations"] == 1 and st["sigma_vectors"] > 0
    assert np.isfinite(e).all() and np.all(np.diff(e) >= 0)
    assert np.isfinite(p).all()
    assert np.isfinite(vec).all() and (np.abs(vec).max(axis=1) > 0).all()
    assert st["max_residual"] > 1e-4  # one iteration does not converge this system


def test_nan_mlp_weights_fall_back_to_diagonal():
    from paper_2012_06714_gb300 import ADC, mlp_nweights

    s = _system()
    ref = ADC(s.eps, s.B, 4, order=3, kind="ea", precision="fp64", res_tol=1e-6)
    e0, p0, _, st0 = ref.davidson(3, tol=1e-9)
    ref.close()
    g = ADC(s.eps, s.B, 4, order=3, kind="ea", precision="fp64", res_tol=1e-6)
    g.set_mlp(np.full(mlp_nweights(), np.nan, dtype=np.float32))
    e, p, _, st = g.davidson(3, tol=1e-9)
    g.close()
    assert st0["status"] == 0 and st["status"] == 0
    assert st["mlp_fallbacks"] == 3
    assert np.abs(e - e0).max() < 1e-8
    assert np.abs(p - p0).max() < 1e-6


def test_nan_in_guess_is_rejected():
    from paper_2012_06714_gb300 import ADC
    from paper_2012_06714_gb300._lib import ADCError

    s = _system()
    g = ADC(s.eps, s.B, 4, order=2, kind="ip", precision="fp64")
    guess = np.zeros((2, g.dim))
    guess[0, 0] = guess[1, 1] = 1.0
    guess[1, 5] = np.nan
    with pytest.raises(ADCError) as ex:
        g.davidson(2, tol=1e-8, guess=guess)
    assert ex.value.code == NONFINITE
    # the handle stays usable after the failed call
    e, _, _, st = g.davidson(2, tol=1e-8)
    assert st["status"] == 0 and np.isfinite(e).all()
    g.close()


def test_nonfinite_sigma_stops_the_solver():
    from paper_2012_06714_gb300 import ADC
    from paper_2012_06714_gb300._lib import ADCError

    s = _system()
    eps = s.eps.copy()
    eps[6] = np.nan  # a virtual orbital energy
    g = ADC(eps, s.B, 4, order=2, kind="ea", precision="fp64")
    with pytest.raises(ADCError) as ex:
        g.davidson(2, tol=1e-8)
    assert ex.value.code == NONFINITE
    g.close()
