"""The kernel-timing hook (adr_profile_kernel / adr_profile_read) and the launch counter.

Timing a kernel class must not change a single bit of the solve, and every
class must see launches in a 3-level K-cycle solve.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _problem():
    from paper_1712_06091_gb300 import workloads as W
    return W.constant_medium((33, 33, 17), src=(16, 16, 2))


def _operator(P, **kw):
    import torch
    from paper_1712_06091_gb300 import adr as gpu
    params = gpu.default_params(levels=3, **kw)
    return gpu.Operator(P.n, P.h, P.src, P.omega, torch.from_numpy(P.kappa), torch.from_numpy(P.tau1),
                        torch.from_numpy(P.gamma),
                        params=params)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_profile_is_transparent(adrlib, cuda, precision):
    from paper_1712_06091_gb300 import adr as gpu
    P = _problem()
    with _operator(P, precision=precision) as op:
        a0, i0 = op.solve(tol=1e-8, maxit=200)
        a0 = a0.cpu().numpy()
        for cls in ("level1_relax", "fine_relax", "outer_apply", "coarsest"):
            op.profile(cls)
            before = gpu.kernel_launches()
            a1, i1 = op.solve(tol=1e-8, maxit=200)
            launched = gpu.kernel_launches() - before
            count, ms = op.profile_read()
            assert i1["iterations"] == i0["iterations"]
            assert np.array_equal(a1.cpu().numpy(), a0), cls
            assert count > 0 and ms > 0.0, (cls, count, ms)
            assert launched > 0
            if cls in ("level1_relax", "coarsest"):
                # one preconditioner application per FGMRES iteration
                assert count % i1["iterations"] == 0, (cls, count, i1["iterations"])
        # re-enabling the same class keeps the captured cycle and restarts the totals
        op.profile("coarsest")
        a2, i2 = op.solve(tol=1e-8, maxit=200)
        count, ms = op.profile_read()
        assert np.array_equal(a2.cpu().numpy(), a0)
        assert count > 0 and count % i2["iterations"] == 0 and ms > 0.0
        op.profile("none")
        op.solve(tol=1e-8, maxit=200)
        count, ms = op.profile_read()
        assert count == 0 and ms == 0.0


def test_profile_rejects_unknown_class(adrlib, cuda):
    from paper_1712_06091_gb300 import _lib as L
    P = _problem()
    with _operator(P) as op:
        rc = L.load().adr_profile_kernel(op._h, 99)
        assert rc == L.ADR_ERR_ARG
