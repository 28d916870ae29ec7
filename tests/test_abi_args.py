"""Argument validation of the C ABI on the host: every invalid parameter is
rejected with ADR_ERR_ARG and a message naming it, before any device work,
so these run without a GPU (the array pointers are never dereferenced)."""
import ctypes

import pytest

DUMMY = ctypes.c_void_p(16)   # never dereferenced: validation fails first

# (field, invalid value, word expected in the message)
BAD_PARAMS = [
    ("levels", 0, "levels"), ("levels", 9, "levels"),
    ("beta", -0.5, "beta"), ("beta", 1.5, "beta"),
    ("cycle", 7, "cycle"), ("relax", 5, "relaxation"),
    ("coarse_iterations", 0, "coarse_iterations"), ("kcycle_iterations", 17, "kcycle_iterations"),
    ("restart", 65, "restart"), ("precond_precision", 3, "precision"),
    ("near_source", 0, "near_source"), ("reorth_eta", -1.0, "reorth_eta"),
    ("adjoint", 2, "adjoint"), ("relax_blocks", -1, "relax_blocks"), ("relax_blocks", 10241, "relax_blocks"),
    ("coarse_solver", 99, "coarse_solver"), ("tma", 5, "tma"),
    ("scheme", 3, "scheme"), ("prec_scheme", 9, "prec_scheme"), ("rescale", 2, "rescale"),
    ("kcycle_threshold", -0.1, "kcycle_threshold"), ("kcycle_threshold", float("nan"), "kcycle_threshold"),
    ("outer_df", 2, "outer_df"),
]


def _grid():
    n = (ctypes.c_int * 3)(9, 9, 1)
    h = (ctypes.c_double * 3)(0.1, 0.1, 1.0)
    s = (ctypes.c_int * 3)(4, 4, 0)
    return n, h, s


@pytest.mark.parametrize("field,value,word", BAD_PARAMS)
def test_invalid_parameter_rejected(adrlib, field, value, word):
    from paper_1712_06091_gb300 import _lib
    p = _lib.Params()
    assert adrlib.adr_params_default(ctypes.byref(p)) == _lib.ADR_OK
    setattr(p, field, value)
    n, h, s = _grid()
    out = ctypes.c_void_p()
    rc = adrlib.adr_operator_create(2, n, h, s, 1.0, DUMMY, DUMMY, DUMMY, ctypes.byref(p), None, ctypes.byref(out))
    assert rc == _lib.ADR_ERR_ARG, (field, value, rc)
    assert word.encode() in adrlib.adr_last_error(), adrlib.adr_last_error()
    assert not out.value


@pytest.mark.parametrize("field", ["pre_sweeps", "post_sweeps", "jacobi_weight"])
def test_invalid_per_level_parameter_rejected(adrlib, field):
    from paper_1712_06091_gb300 import _lib
    p = _lib.Params()
    assert adrlib.adr_params_default(ctypes.byref(p)) == _lib.ADR_OK
    getattr(p, field)[1] = 17 if field != "jacobi_weight" else 0.0
    n, h, s = _grid()
    out = ctypes.c_void_p()
    rc = adrlib.adr_operator_create(2, n, h, s, 1.0, DUMMY, DUMMY, DUMMY, ctypes.byref(p), None, ctypes.byref(out))
    assert rc == _lib.ADR_ERR_ARG, (field, rc)


@pytest.mark.parametrize("omega,h0", [(0.0, 0.1), (-1.0, 0.1), (1.0, 0.0), (1.0, -0.1)])
def test_invalid_frequency_or_spacing_rejected(adrlib, omega, h0):
    from paper_1712_06091_gb300 import _lib
    n, h, s = _grid()
    h[0] = h0
    out = ctypes.c_void_p()
    rc = adrlib.adr_operator_create(2, n, h, s, omega, DUMMY, DUMMY, DUMMY, None, None, ctypes.byref(out))
    assert rc == _lib.ADR_ERR_ARG


def test_batch_problem_count_rejected(adrlib):
    from paper_1712_06091_gb300 import _lib
    n, h, s = _grid()
    om = (ctypes.c_double * 1)(1.0)
    out = ctypes.c_void_p()
    rc = adrlib.adr_batch_create(2, n, h, 0, s, om, DUMMY, DUMMY, DUMMY, None, None, ctypes.byref(out))
    assert rc == _lib.ADR_ERR_ARG and b"problems" in adrlib.adr_last_error()


def test_static_traveltime_limit_rejected(adrlib):
    """The allocation-free travel time rejects more sweeps than its fixed flag array holds."""
    from paper_1712_06091_gb300 import _lib
    n, h, s = _grid()
    done = ctypes.c_int(-1)
    rc = adrlib.adr_traveltime_static(2, n, h, s, DUMMY, DUMMY, 8193, None, ctypes.byref(done))
    assert rc == _lib.ADR_ERR_ARG and b"max_sweeps" in adrlib.adr_last_error()
    rc = adrlib.adr_traveltime_static(2, n, h, s, DUMMY, DUMMY, 0, None, ctypes.byref(done))
    assert rc == _lib.ADR_ERR_ARG


def test_grid_beyond_31_bit_indices_rejected(adrlib):
    """Node indices are 31-bit: a grid of 2^31 nodes or more is refused before any allocation."""
    from paper_1712_06091_gb300 import _lib
    n = (ctypes.c_int * 3)(2048, 2048, 513)
    h = (ctypes.c_double * 3)(0.01, 0.01, 0.01)
    s = (ctypes.c_int * 3)(1024, 1024, 2)
    out = ctypes.c_void_p()
    rc = adrlib.adr_operator_create(3, n, h, s, 1.0, DUMMY, DUMMY, DUMMY, None, None, ctypes.byref(out))
    assert rc == _lib.ADR_ERR_ARG and b"too large" in adrlib.adr_last_error()


def test_traveltime_invalid_arguments_set_the_error_text(adrlib):
    """Both travel-time entry points report an invalid argument through adr_last_error (no device work)."""
    from paper_1712_06091_gb300 import _lib
    n, h, s = _grid()
    adrlib.adr_params_default(None)                      # leaves an unrelated message behind
    for fn in (adrlib.adr_traveltime, adrlib.adr_traveltime_static):
        rc = fn(2, n, h, s, DUMMY, DUMMY, 0, None, None)
        assert rc == _lib.ADR_ERR_ARG and b"invalid argument" in adrlib.adr_last_error()
        bad = (ctypes.c_int * 3)(99, 99, 0)
        rc = fn(2, n, h, bad, DUMMY, DUMMY, 10, None, None)
        assert rc == _lib.ADR_ERR_ARG and b"invalid grid or source" in adrlib.adr_last_error()
