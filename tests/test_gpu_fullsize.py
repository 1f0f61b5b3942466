"""Parity at the benchmark's full size and launch configuration: EA-ADC(3),
nocc=40, nvir=400, naux=1400, mixed precision (tensor-core BF16x3 ladder), a
block of 4 trial vectors.  The full oracle is out of reach at this size, so
(1) sampled 2p1h rows sigma_{n,i,:,:} are computed by the sampled-row oracle
and compared element by element (tolerance 3e-5 of the row's largest element,
the split-BF16 bound of the mixed-precision tests), and (2) the S-symmetry of
M (x^T S M y = y^T S M x), which holds at any size and involves every block,
is checked to 1e-5 relative."""
import numpy as np
import pytest

from adc_inputs import make_system
from oracle.sampled import sigma_ea_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

O, V, NAUX, NVEC = 40, 400, 1400, 4


@pytest.fixture(scope="module")
def run():
    from paper_2012_06714_gb300 import ADC

    s = make_system(O, V, NAUX, seed=0)
    gpu = ADC(torch.from_numpy(s.eps).cuda(), torch.from_numpy(s.B).cuda(), O, order=3, kind="ea",
              precision="bf16x3")
    X = np.random.default_rng(21).standard_normal((NVEC, gpu.dim)) / np.sqrt(gpu.dim)
    S = gpu.sigma(torch.from_numpy(X).cuda()).cpu().numpy()
    yield s, gpu, X, S
    gpu.close()


def test_sampled_rows(run):
    s, gpu, X, S = run
    for n, rows in ((0, [0, 39]), (3, [17])):
        ref = sigma_ea_rows(s.eps, s.B, O, X[n, :V], X[n, V:].reshape(O, V, V), rows, order=3)
        got = S[n, V:].reshape(O, V, V)[rows]
        for r in range(len(rows)):
            assert np.abs(got[r] - ref[r]).max() <= 3e-5 * np.abs(ref[r]).max(), (n, rows[r])


def _apply_S(x):
    y1, y2 = x[:V], x[V:].reshape(O, V, V)
    return np.concatenate([y1, (2.0 * y2 - y2.transpose(0, 2, 1)).ravel()])


def test_s_symmetry(run):
    s, gpu, X, S = run
    a = X[0] @ _apply_S(S[1])
    b = X[1] @ _apply_S(S[0])
    scale = np.sqrt(abs(X[0] @ _apply_S(S[0])) * abs(X[1] @ _apply_S(S[1])))
    assert abs(a - b) <= 1e-5 * scale, (a, b, scale)
    assert np.isfinite(S).all()
