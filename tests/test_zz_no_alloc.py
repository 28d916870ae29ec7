"""adr_traveltime_static (no allocation, flags in a fixed device array) against adr_traveltime.

Collected last on purpose: it must give the allocating entry point's result
both on a fresh library and after every other test has used the device, and
on two calls in a row (the second call finds the flags the first one left).
"""
import ctypes

import numpy as np
import pytest

from paper_1712_06091_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = 1e-12   # same relaxation, same fixed point: agreement to rounding


def _args(n, h, src):
    dim = len(n)
    nn = (ctypes.c_int * 3)(*n, *([1] * (3 - dim)))
    hh = (ctypes.c_double * 3)(*h, *([1.0] * (3 - dim)))
    ss = (ctypes.c_int * 3)(*src, *([0] * (3 - dim)))
    return dim, nn, hh, ss


def _run(fn, n, h, src, kappa, max_sweeps):
    dim, nn, hh, ss = _args(n, h, src)
    tau1 = torch.full((int(np.prod(n)),), -1.0, dtype=torch.float64, device=kappa.device)
    sweeps = ctypes.c_int(-1)
    stream = torch.cuda.current_stream(kappa.device).cuda_stream
    rc = fn(dim, nn, hh, ss, ctypes.c_void_p(kappa.data_ptr()), ctypes.c_void_p(tau1.data_ptr()), int(max_sweeps),
            ctypes.c_void_p(stream), ctypes.byref(sweeps))
    torch.cuda.synchronize()
    return rc, tau1.cpu().numpy(), sweeps.value


CASES = {
    "const2d_33x17": lambda: (W.constant_medium((33, 17), src=(16, 0)), 0.7),
    "marine2d_65x33": lambda: (W.marine_2d((65, 33)), None),
    "layered3d_33x33x17": lambda: (W.layered_3d((33, 33, 17)), None),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_static_matches_allocating_entry_twice(adrlib, cuda, name):
    from paper_1712_06091_gb300 import _lib as L
    P, k0 = CASES[name]()
    kappa_np = np.full(P.N, k0) if k0 is not None else P.kappa
    kappa = torch.from_numpy(np.ascontiguousarray(kappa_np, dtype=np.float64)).to("cuda:0")
    limit = 8 * sum(P.n) + 64
    rc, ref, sweeps_ref = _run(adrlib.adr_traveltime, P.n, P.h, P.src, kappa, limit)
    assert rc == L.ADR_OK and sweeps_ref > 0
    for call in range(2):
        rc, got, sweeps = _run(adrlib.adr_traveltime_static, P.n, P.h, P.src, kappa, limit)
        assert rc == L.ADR_OK, (call, adrlib.adr_last_error())
        assert sweeps > 0
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0.0, err_msg=f"call {call}")


def test_static_rejects_more_sweeps_than_its_array(adrlib, cuda):
    from paper_1712_06091_gb300 import _lib as L
    P = W.constant_medium((9, 9), src=(4, 4))
    kappa = torch.ones(P.N, dtype=torch.float64, device="cuda:0")
    rc, got, _ = _run(adrlib.adr_traveltime_static, P.n, P.h, P.src, kappa, L.TRAVELTIME_STATIC_MAX_SWEEPS + 1)
    assert rc == L.ADR_ERR_ARG
    assert b"8192" in adrlib.adr_last_error()
    assert np.all(got == -1.0)       # rejected before any device work
    rc, got, _ = _run(adrlib.adr_traveltime_static, P.n, P.h, P.src, kappa, L.TRAVELTIME_STATIC_MAX_SWEEPS)
    assert rc == L.ADR_OK and np.allclose(got, 1.0, rtol=1e-12)
