"""Device travel-time factor (adr_traveltime) against closed forms and the oracle's fast marching."""
import math

import numpy as np
import pytest

from oracle import adr, eikonal
from paper_1712_06091_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n,src", [((33, 17), (16, 0)), ((13, 11, 9), (0, 5, 8))])
def test_constant_medium_exact(adrlib, cuda, n, src):
    from paper_1712_06091_gb300 import adr as gpu
    h = tuple(0.05 * (d + 1) for d in range(len(n)))
    kappa = np.full(int(np.prod(n)), 0.7)
    tau1, sweeps = gpu.traveltime(n, h, src, kappa)
    assert np.abs(tau1.cpu().numpy() - 0.7).max() < 1e-12 and sweeps > 0


def test_linear_gradient_first_order_and_matches_fast_marching(adrlib, cuda):
    from paper_1712_06091_gb300 import adr as gpu
    errs = []
    for n in (65, 129, 257):
        nn = (n, (n + 1) // 2)
        src = ((nn[0] - 1) // 2, 2)
        P = W.linear_velocity(nn, (2.0, 1.0), 1.5, 1.0, src)
        ref = W.linear_velocity_traveltime(P.n, P.h, src, 1.5, 1.0)
        t1, _ = gpu.traveltime(P.n, P.h, src, P.kappa)
        g = adr.Grid(P.n, P.h)
        tau0 = adr.travel_time(g, src, np.ones(g.N))
        t1 = t1.cpu().numpy()
        errs.append(np.abs((t1 - ref) * tau0).max())
        if n == 65:
            fm = eikonal.factored_fast_marching(g, P.kappa, src, order=1)
            # same first-order upwind system, different solution order: agree to well below its error
            assert np.abs((fm - t1) * tau0).max() < 0.2 * errs[0]
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 0.75, (errs, rates)


@pytest.mark.parametrize("n,src", [((33, 17), (16, 0)), ((13, 11, 9), (0, 5, 8))])
def test_second_order_constant_medium_exact(adrlib, cuda, n, src):
    from paper_1712_06091_gb300 import adr as gpu
    h = tuple(0.05 * (d + 1) for d in range(len(n)))
    kappa = np.full(int(np.prod(n)), 0.7)
    tau1, sweeps = gpu.traveltime(n, h, src, kappa, order=2)
    assert np.abs(tau1.cpu().numpy() - 0.7).max() < 1e-12 and sweeps > 0


def test_second_order_converges_like_fast_marching(adrlib, cuda):
    """The second-order device update (Sec. 2.1's factored fast marching with
    second-order differences) converges at the rate of the oracle's order-2
    fast marching in the linear velocity gradient (textbook travel time), and
    the two agree to a fraction of that error."""
    from paper_1712_06091_gb300 import adr as gpu
    errs, errs_fm = [], []
    for n in (33, 65, 129):
        nn = (n, (n + 1) // 2)
        src = ((nn[0] - 1) // 2, 2)
        P = W.linear_velocity(nn, (2.0, 1.0), 1.5, 1.0, src)
        ref = W.linear_velocity_traveltime(P.n, P.h, src, 1.5, 1.0)
        t1, _ = gpu.traveltime(P.n, P.h, src, P.kappa, order=2)
        g = adr.Grid(P.n, P.h)
        tau0 = adr.travel_time(g, src, np.ones(g.N))
        t1 = t1.cpu().numpy()
        fm = eikonal.factored_fast_marching(g, P.kappa, src, order=2)
        errs.append(np.abs((t1 - ref) * tau0).max())
        errs_fm.append(np.abs((fm - ref) * tau0).max())
        assert np.abs((fm - t1) * tau0).max() < 0.5 * errs_fm[-1], (n, np.abs((fm - t1) * tau0).max(), errs_fm[-1])
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 1.6, (errs, rates, errs_fm)
    assert errs[-1] < 2.0 * errs_fm[-1]


def test_second_order_3d_layered(adrlib, cuda):
    """3D: the device order-2 travel time is close to the oracle's order-2 fast
    marching on the layered model and at least as close to it as order 1."""
    from paper_1712_06091_gb300 import adr as gpu
    P = W.layered_3d((17, 17, 9))
    g = adr.Grid(P.n, P.h)
    fm = eikonal.factored_fast_marching(g, P.kappa, P.src, order=2)
    t2 = gpu.traveltime(P.n, P.h, P.src, P.kappa, order=2)[0].cpu().numpy()
    t1 = gpu.traveltime(P.n, P.h, P.src, P.kappa)[0].cpu().numpy()
    tau0 = adr.travel_time(g, P.src, np.ones(g.N))
    e2, e1 = np.abs((t2 - fm) * tau0).max(), np.abs((t1 - fm) * tau0).max()
    assert e2 < e1 and e2 < 1e-3 * np.abs(fm * tau0).max(), (e2, e1)
