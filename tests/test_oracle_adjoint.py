"""Pins of the oracle's adjoint-state gradient (no GPU): central finite
differences of the misfit itself, with direct solves, along random directions
supported on random node subsets; and the sign/scale of the misfit at the data."""
import numpy as np
import pytest

from oracle import adjoint, adr, eikonal
from paper_1712_06091_gb300 import workloads as W


def _problem(n=(33, 17), nsrc=2, seed=7):
    P = W.marine_2d(n)
    g = adr.Grid(P.n, P.h)
    rng = np.random.default_rng(seed)
    sources = [(int(x), 1) for x in rng.choice(np.arange(4, n[0] - 4), size=nsrc, replace=False)]
    tau1s = [eikonal.factored_fast_marching(g, P.kappa, s, order=2) for s in sources]
    receivers = np.array([i + n[0] * 0 for i in range(2, n[0] - 2, 4)], dtype=np.int64)   # top row
    # data from a slightly different slowness, so that the misfit is not at its minimum
    kappa_true = P.kappa * (1.0 + 0.02 * W.smooth_random_field(P.n, seed=11))
    data = []
    for s, t1 in zip(sources, tau1s):
        _, _, u = adjoint.forward_wavefield(g, s, P.omega, kappa_true, P.gamma, t1)
        data.append(u[receivers])
    return P, g, sources, tau1s, receivers, data


def test_gradient_matches_central_differences():
    P, g, sources, tau1s, rec, data = _problem()
    J, grad = adjoint.misfit_gradient(g, sources, P.omega, P.kappa, P.gamma, tau1s, rec, data)
    assert J > 0.0
    rng = np.random.default_rng(3)
    for trial in range(4):
        v = np.zeros(g.N)
        subset = rng.choice(g.N, size=g.N // 8, replace=False)
        v[subset] = rng.standard_normal(subset.size) * P.kappa[subset]
        eps = 1e-6
        Jp = adjoint.misfit(g, sources, P.omega, P.kappa + eps * v, P.gamma, tau1s, rec, data)
        Jm = adjoint.misfit(g, sources, P.omega, P.kappa - eps * v, P.gamma, tau1s, rec, data)
        fd = (Jp - Jm) / (2 * eps)
        an = float(grad @ v)
        assert abs(fd - an) <= 1e-6 * abs(an), (trial, fd, an)


def test_misfit_vanishes_at_the_data_and_gradient_with_it():
    P, g, sources, tau1s, rec, _ = _problem(nsrc=1)
    data = [adjoint.forward_wavefield(g, sources[0], P.omega, P.kappa, P.gamma, tau1s[0])[2][rec]]
    J, grad = adjoint.misfit_gradient(g, sources, P.omega, P.kappa, P.gamma, tau1s, rec, data)
    assert J < 1e-25 * max(1.0, float(np.abs(data[0]).max()) ** 2)
    assert np.abs(grad).max() < 1e-10
