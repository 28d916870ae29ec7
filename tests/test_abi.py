"""The C-ABI library loads without a GPU and exports every entry point that
include/adr.h declares; argument checks fail cleanly before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "adr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(adr_[a-z0-9_]+)\s*\(", text)))


def test_header_and_binding_agree(adrlib):
    from paper_1712_06091_gb300 import _lib
    declared = _declared()
    assert declared == sorted(_lib.EXPORTS)
    for name in declared:
        assert hasattr(adrlib, name), name


def test_defaults_and_argument_errors(adrlib):
    from paper_1712_06091_gb300 import _lib
    p = _lib.Params()
    assert adrlib.adr_params_default(ctypes.byref(p)) == 0
    assert (p.levels, p.beta, p.cycle, p.relax, p.coarse_iterations, p.kcycle_iterations) == (5, 0.25, 1, 1, 10, 2)
    assert list(p.pre_sweeps)[:5] == [2, 3, 4, 5, 6]
    assert p.near_source == 1
    out = ctypes.c_void_p()
    n = (ctypes.c_int * 3)(9, 9, 1)
    h = (ctypes.c_double * 3)(0.1, 0.1, 1.0)
    s = (ctypes.c_int * 3)(4, 4, 0)
    dummy = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    rc = adrlib.adr_operator_create(4, n, h, s, 1.0, dummy, dummy, dummy, None, None, ctypes.byref(out))
    assert rc == _lib.ADR_ERR_ARG and b"dim" in adrlib.adr_last_error()
    s_bad = (ctypes.c_int * 3)(9, 4, 0)
    rc = adrlib.adr_operator_create(2, n, h, s_bad, 1.0, dummy, dummy, dummy, None, None, ctypes.byref(out))
    assert rc == _lib.ADR_ERR_ARG and b"source" in adrlib.adr_last_error()
    n_small = (ctypes.c_int * 3)(3, 9, 1)
    rc = adrlib.adr_operator_create(2, n_small, h, s, 1.0, dummy, dummy, dummy, None, None, ctypes.byref(out))
    assert rc == _lib.ADR_ERR_ARG
    p.restart = 0
    rc = adrlib.adr_operator_create(2, n, h, s, 1.0, dummy, dummy, dummy, ctypes.byref(p), None, ctypes.byref(out))
    assert rc == _lib.ADR_ERR_ARG and b"restart" in adrlib.adr_last_error()
    assert adrlib.adr_params_default(ctypes.byref(p)) == 0 and p.shift == 0.0
    for bad in (-0.1, float("nan"), 101.0):
        p.shift = bad
        rc = adrlib.adr_operator_create(2, n, h, s, 1.0, dummy, dummy, dummy, ctypes.byref(p), None, ctypes.byref(out))
        assert rc == _lib.ADR_ERR_ARG and b"shift" in adrlib.adr_last_error()
    assert adrlib.adr_version() == b"0.1.0"
