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
