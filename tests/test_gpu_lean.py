"""The memory-lean layout (adc_options.lean = 1) of a closed-shell EA handle in
mixed precision: the o^2 v^2 integrals and amplitudes held in FP32, no tau or
ring2 tensor (their contractions expanded into ones with t and the integrals),
operand copies made per call, setup temporaries in FP32, and the transition
moments' root-independent parts made at setup.  It is the layout that lets the
1028-MO workload fit one GPU; here it is checked at sizes the oracle reaches.

Bars: sigma against the FP64 oracle at the mixed-precision tolerance of the
plain layout (3e-5 of max |sigma|, see test_gpu_mixed); lean against plain
sigma at 1e-5 of max |sigma| (the two differ only by FP32 storage of operands
that both split into the same BF16 planes, and by the order of the expanded
tau / ring2 terms); t2 is the FP32 rounding of the plain handle's (2^-24
relative), t2(2) within 1e-6 relative (its ring terms accumulate in FP32);
E(2) identical, E(3) within 1e-9 Eh; the roots and spectroscopic factors at
nocc 20, nvir 180, naux 600 against the stored oracle roots at the mixed
path's bars, 1e-6 Eh and 1e-6."""
import json
import os

import numpy as np
import pytest

from adc_inputs import make_system
from oracle.spinadapted import SpinAdaptedADC

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(4, 14, 40, 0), (6, 70, 150, 1)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"o{c[0]}v{c[1]}Q{c[2]}")
def test_sigma_lean_vs_oracle_and_plain(case):
    from paper_2012_06714_gb300 import ADC

    o, v, naux, seed = case
    s = make_system(o, v, naux, seed=seed)
    lean = ADC(s.eps, s.B, o, order=3, kind="ea", precision="bf16x3", lean=1)
    plain = ADC(s.eps, s.B, o, order=3, kind="ea", precision="bf16x3", lean=0)
    ref = SpinAdaptedADC(s.eps, o, s.B, 3, "ea")
    X = np.random.default_rng(5).standard_normal((3, lean.dim))
    Sl, Sp, Sr = lean.sigma(X), plain.sigma(X), ref.sigma(X)
    L = np.abs(ref.ladder(X[:, v:].reshape(3, o, v, v))).max()
    scale = max(L, np.abs(Sr).max())
    assert np.isfinite(Sl).all()
    assert np.abs(Sl - Sr).max() <= 3e-5 * scale, np.abs(Sl - Sr).max() / scale
    assert np.abs(Sl - Sp).max() <= 1e-5 * np.abs(Sp).max(), np.abs(Sl - Sp).max() / np.abs(Sp).max()
    # setup tensors
    t_l, t_p = lean.get("t2", (o, o, v, v)), plain.get("t2", (o, o, v, v))
    assert np.abs(t_l - t_p).max() <= 2.0 ** -24 * np.abs(t_p).max()
    u_l, u_p = lean.get("t2_2", (o, o, v, v)), plain.get("t2_2", (o, o, v, v))
    assert np.abs(u_l - u_p).max() <= 1e-6 * np.abs(u_p).max()
    e_l, e_p = lean.mp_energy(), plain.mp_energy()
    assert abs(e_l[0] - e_p[0]) <= 1e-12 * abs(e_p[0])
    assert abs(e_l[1] - e_p[1]) <= 1e-9
    lean.close()
    plain.close()


def test_lean_roots_match_stored_oracle_roots():
    from paper_2012_06714_gb300 import ADC

    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cfg1_roots.json")))
    g = gold["system"]
    s = make_system(g["nocc"], g["nvir"], g["naux"], seed=g["seed"])
    ref = gold["ea"]
    n = len(ref["energies_eh"])
    h = ADC(s.eps, s.B, s.nocc, order=3, kind="ea", precision="bf16x3", max_iter=300, max_space_per_root=12,
            res_tol=3e-5, refine_res_tol=1e-6, lean=1)
    e, p, _, st = h.davidson(n, tol=1e-8)
    h.close()
    assert st["status"] == 0
    de = np.abs(e - np.array(ref["energies_eh"])).max()
    dp = np.abs(p - np.array(ref["spectroscopic_factors"])).max()
    print(f"lean ea bf16x3: max |dE| {de:.2e} Eh, max |dP| {dp:.2e}, residual {st['max_residual']:.1e}")
    assert de <= 1e-6, de
    assert dp <= 1e-6, dp


@pytest.mark.parametrize("kw", [dict(kind="ip", precision="bf16x3"), dict(kind="ea", precision="fp64"),
                                dict(kind="ea", precision="bf16x3", m11_on_the_fly=1)])
def test_lean_refused_where_it_does_not_apply(kw):
    from paper_2012_06714_gb300 import ADC
    from paper_2012_06714_gb300._lib import ADCError

    s = make_system(3, 10, 30, seed=2)
    with pytest.raises(ADCError):
        ADC(s.eps, s.B, 3, order=3, lean=1, **kw)
