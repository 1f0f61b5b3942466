"""Training samples for the learned Davidson preconditioner (adc_mlp_train).

The samples come from the library (adc_mlp_samples): the handle's own plain
Davidson iterates, their residuals and the exact corrections are formed on the
device; this module only forwards the arguments.
"""
from __future__ import annotations


def davidson_samples(adc, nroots, iters=(1, 2, 3, 4, 6, 8, 10, 14), per_vector=100_000, seed=0, exact_tol=1e-10):
    """(d, blk, r, t) sample arrays from the Davidson trajectory of `adc` (an ADC handle)."""
    return adc.mlp_samples(nroots, iters=iters, per_vector=per_vector, seed=seed, exact_tol=exact_tol)
