"""The C ABI library builds for sm_103a, loads, and exports every function that
include/adc.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "adc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(adc_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2012_06714_gb300 import build_library, library_path

    if not os.path.exists(library_path()):
        build_library()
    return ctypes.CDLL(library_path())


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("adc_setup", "adc_sigma", "adc_davidson", "adc_dim", "adc_destroy", "adc_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_loads(lib):
    from paper_2012_06714_gb300 import load_library
    from paper_2012_06714_gb300._lib import EXPORTED

    L = load_library()
    assert set(EXPORTED) <= set(declared_functions())


def test_default_options_and_argument_errors(lib):
    from paper_2012_06714_gb300._lib import Options, load_library

    L = load_library()
    o = Options()
    assert L.adc_default_options(ctypes.byref(o)) == 0
    assert o.precision == 0 and o.max_space_per_root == 8 and o.max_iter == 100
    assert o.refine == 1 and o.transition_order == 0 and o.contractions == -1
    assert L.adc_default_options(None) == -1
    h = ctypes.c_void_p()
    # invalid sizes are rejected on the host before any device work
    assert L.adc_setup(None, None, 0, 5, 5, 3, 1, None, 0, ctypes.byref(h)) == -1
    assert b"invalid" in L.adc_last_error(None)
    assert L.adc_dim(None, None) == -1
