"""The allocation-free ladder entry point (adc_ladder_noalloc), through the C ABI.

It serves callers that cannot allocate device memory during a call (their own
memory manager owns the device memory and forbids cudaMalloc/cudaFree inside
library calls).  Its output must equal that of the existing entry point
adc_sigma: with B^Q_oo = B^Q_ov = 0 every amplitude, ring and coupling term of
EA-ADC(3) vanishes and the 2p1h block is exactly diag + ladder, so
ladder(Y) = sigma_2p1h(0 + Y) - diag * Y.  Two calls in a row are checked (the
fixed scratch keeps the previous call's contents).  Tolerance: the 3e-5
split-BF16 bound of the mixed-precision tests, relative to max |ladder|.
This file is collected last."""
import ctypes

import numpy as np
import pytest

from adc_inputs import make_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _vv_only_system(o, v, naux, seed):
    s = make_system(o, v, naux, seed=seed)
    B = s.B.copy()
    B[:, :o, :] = 0.0
    B[:, :, :o] = 0.0
    return s.eps, B


# (nocc, nvir, naux, nvec): the first fits in one group of matrices and one auxiliary chunk;
# in the second (12 matrices of 400 x 400) the 64 MiB holds 11 matrices' split X^T and Z,
# so the matrices run in two groups and the 100 auxiliary functions in 13 chunks of 8.
CASES = [(3, 70, 61, 2), (4, 400, 100, 3)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"o{c[0]}v{c[1]}Q{c[2]}n{c[3]}")
def test_noalloc_ladder_matches_sigma_twice(case):
    from paper_2012_06714_gb300 import ADC

    o, v, naux, nvec = case
    eps, B = _vv_only_system(o, v, naux, 4)
    gpu = ADC(eps, B, o, order=3, kind="ea", precision="bf16x3")
    dim = gpu.dim
    rng = np.random.default_rng(11)
    X = rng.standard_normal((nvec, dim))
    X[:, :v] = 0.0
    S = gpu.sigma(X)
    diag = gpu.get("diag", (dim,))
    ref = (S[:, v:] - diag[v:] * X[:, v:]).reshape(nvec * o, v, v)
    Xd = torch.from_numpy(np.ascontiguousarray(X[:, v:].reshape(nvec * o, v, v))).cuda()
    lib = gpu._lib
    scale = np.abs(ref).max()
    for call in range(2):
        out = torch.full((nvec * o, v, v), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.adc_ladder_noalloc(gpu._h, ctypes.c_void_p(Xd.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_longlong(nvec * o))
        assert rc == 0, lib.adc_last_error(gpu._h)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 3e-5 * scale, (call, np.abs(got - ref).max(), scale)
    gpu.close()


def test_noalloc_ladder_rejects_fp64_handle():
    from paper_2012_06714_gb300 import ADC

    eps, B = _vv_only_system(2, 20, 12, 1)
    gpu = ADC(eps, B, 2, order=3, kind="ea", precision="fp64")
    x = torch.zeros((2, 20, 20), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    rc = gpu._lib.adc_ladder_noalloc(gpu._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                     ctypes.c_longlong(2))
    assert rc == -1
    assert b"BF16X3" in gpu._lib.adc_last_error(gpu._h)
    gpu.close()
