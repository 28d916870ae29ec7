"""Pins of the oracle's ADR discretisation against facts the paper and the
mathematics fix (no GPU).

* hand-derived rows (tests/golden/adr_rows_2d.txt: Eqs. ADR, londUpwindDiff,
  1up, precADRup, BCADR, helmADR2);
* tau = 0 turns every ADR matrix into the standard Helmholtz matrix
  (Sec. 1: "if we choose tau = 0 ... a = u");
* M^{-1} H M and H_cen / H_2up differ by O(h^2) at fixed omega, H_1up by O(h)
  (Eq. matrix_rescaling and the expansion of Eqs. helmADR2-helmADR4);
* the travel-time coefficient formulas (Eq. travel_time_coeff) on fields with
  known derivatives.
"""
import math
import os

import numpy as np
import pytest

from oracle import adr
from paper_1712_06091_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "adr_rows_2d.txt")


def _golden_setting():
    n, h, src = (9, 9), (0.1, 0.2), (4, 4)
    g = adr.Grid(n, h)
    N = g.N
    return g, src, 2.0, np.ones(N), np.zeros(N), np.ones(N)


def test_golden_rows():
    g, src, omega, kappa, gamma, tau1 = _golden_setting()
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            sch, r0, r1, c0, c1, re, im = line.split()
            rows.setdefault((sch, int(r0), int(r1)), {})[(int(c0), int(c1))] = complex(float(re), float(im))
    assert len(rows) == 5
    for (sch, r0, r1), expect in rows.items():
        j = g.index((r0, r1))
        if sch == "prec":
            A = adr.assemble_preconditioner(g, src, omega, kappa, gamma, tau1, beta=0.25)
            got = {g.coords(int(c)): v for c, v in zip(A[j].indices, A[j].data) if v != 0}
        else:
            got = {g.coords(c): v for c, v in adr.adr_row(g, src, omega, kappa, gamma, tau1, j, sch).items() if v != 0}
        expect = {k: v for k, v in expect.items() if v != 0}
        assert set(got) == set(expect), (sch, r0, r1, sorted(got), sorted(expect))
        for k, v in expect.items():
            assert abs(got[k] - v) <= 1e-12 * max(1.0, abs(v)), (sch, r0, r1, k, got[k], v)


@pytest.mark.parametrize("n,h,src", [((13, 9), (0.1, 0.07), (6, 0)), ((7, 6, 5), (0.2, 0.1, 0.15), (0, 5, 2))])
def test_tau_zero_gives_helmholtz(n, h, src):
    """tau1 = 0 => tau = 0 => every ADR matrix equals H, ghosts and source row included."""
    g = adr.Grid(n, h)
    rng = np.random.default_rng(5)
    kappa = 1.0 + 0.3 * rng.random(g.N)
    gamma = 2.0 * rng.random(g.N)
    omega = 3.7
    H = adr.assemble_helmholtz(g, omega, kappa, gamma).toarray()
    for scheme in ("2up", "1up", "cen"):
        A = adr.assemble_adr(g, src, omega, kappa, gamma, np.zeros(g.N), scheme).toarray()
        assert np.array_equal(A, H), scheme


def _smooth_amplitude(grid, src):
    """A smooth test amplitude a(x) (no singularity)."""
    X = W.node_coordinates(grid.n, grid.h)
    a = np.ones(grid.N, dtype=np.complex128)
    for d, x in enumerate(X):
        a = a * (1.0 + 0.3 * np.cos(1.3 * x + d) + 0.2j * np.sin(0.7 * x - d))
    return a


def _interior_mask(grid, src, margin_frac=0.25, radius=0.3):
    """Rows away from the boundary and at least `radius` (physical) from the source:
    the expansion of Eq. helmADR3 is uniform only at a fixed distance from x0,
    where the derivatives of tau stay bounded as h -> 0."""
    idx = [np.arange(grid.N) // grid.stride[d] % grid.n[d] for d in range(grid.dim)]
    m = np.ones(grid.N, dtype=bool)
    for d in range(grid.dim):
        lo = int(margin_frac * (grid.n[d] - 1))
        m &= (idx[d] >= lo) & (idx[d] <= grid.n[d] - 1 - lo)
    r = np.sqrt(sum(((idx[d] - src[d]) * grid.h[d]) ** 2 for d in range(grid.dim)))
    return m & (r >= radius)


def _rescaling_gap(n, extent, scheme, dim):
    """max over interior rows of |(H_hat - M^{-1} H M) a| / |H_hat a| for exact tau = r."""
    h = tuple(e / (v - 1) for e, v in zip(extent, n))
    g = adr.Grid(n, h)
    src = tuple((v - 1) // 4 for v in n)      # off-centre source inside the grid
    kappa = np.ones(g.N)
    gamma = np.zeros(g.N)
    tau1 = np.ones(g.N)
    omega = 6.0
    A = adr.assemble_adr(g, src, omega, kappa, gamma, tau1, scheme)
    H = adr.assemble_helmholtz(g, omega, kappa, gamma)
    M = adr.phase_matrix(g, src, omega, tau1)
    Minv = adr.phase_matrix(g, src, -omega, tau1)
    a = _smooth_amplitude(g, src)
    mask = _interior_mask(g, src)
    lhs = (A @ a)[mask]
    ref = (Minv @ (H @ (M @ a)))[mask]
    return np.max(np.abs(lhs - ref)) / np.max(np.abs(ref))


@pytest.mark.parametrize("scheme,order", [("cen", 2), ("2up", 2), ("1up", 1)])
def test_rescaling_relation_2d(scheme, order):
    """Eq. matrix_rescaling: M^{-1} H M ~ H_hat with an O(h^order) gap at fixed omega.

    Anisotropic spacing and a non-square grid pin the axis bookkeeping; a dropped
    term (Delta-tau averaging, advection) or a wrong sign leaves an O(1) gap."""
    gaps = [_rescaling_gap((n, (n + 1) // 2 + 4), (2.0, 1.3), scheme, 2) for n in (41, 81, 161)]
    rates = [math.log2(gaps[k] / gaps[k + 1]) for k in range(2)]
    assert gaps[-1] < 0.05
    assert min(rates) > order - 0.35, (gaps, rates)


def test_rescaling_relation_3d():
    gaps = [_rescaling_gap((n, n - 2, (n + 1) // 2 + 2), (1.0, 0.9, 0.6), "2up", 3) for n in (17, 33)]
    assert gaps[1] < gaps[0] / 3.0, gaps


def test_upwind_side_follows_the_wave():
    """Eq. londUpwindDiff: with the source at the left, a node to its right couples to
    j-2 (upwind side), never to j+2; central advection within one node of the source."""
    g = adr.Grid((15, 11), (0.1, 0.1))
    src = (3, 5)
    N = g.N
    row = adr.adr_row(g, src, 5.0, np.ones(N), np.zeros(N), np.ones(N), g.index((9, 5)), "2up")
    assert g.index((7, 5)) in row and g.index((11, 5)) not in row
    row = adr.adr_row(g, src, 5.0, np.ones(N), np.zeros(N), np.ones(N), g.index((1, 5)), "2up")
    assert g.index((3, 5)) in row and abs(row[g.index((3, 5))]) > 0
    near = adr.adr_row(g, src, 5.0, np.ones(N), np.zeros(N), np.ones(N), g.index((4, 6)), "2up")
    assert g.index((6, 6)) not in near and g.index((2, 6)) not in near


def test_coefficients_known_fields():
    """Eq. travel_time_coeff on tau1 = quadratic polynomial: central differences are exact
    inside, the one-sided second derivative is exact on the boundary."""
    n, h = (9, 8), (0.25, 0.2)
    g = adr.Grid(n, h)
    X = W.node_coordinates(n, h)
    c = (0.3, -0.2, 0.15, 0.05, -0.1)
    tau1 = 1.0 + c[0] * X[0] + c[1] * X[1] + c[2] * X[0] ** 2 + c[3] * X[1] ** 2 + c[4] * X[0] * X[1]
    src = (2, 3)
    for j in range(g.N):
        i = g.coords(j)
        x0, x1 = X[0][j], X[1][j]
        d1 = [c[0] + 2 * c[2] * x0 + c[4] * x1, c[1] + 2 * c[3] * x1 + c[4] * x0]
        d2 = [2 * c[2], 2 * c[3]]
        for d in range(2):
            fd = adr.tau1_first_derivative(g, tau1, i, d)
            if 0 < i[d] < n[d] - 1:
                assert abs(fd - d1[d]) < 1e-12
            else:   # first-order one-sided: exact slope of the chord
                k = i[d]
                other = (1 if k == 0 else n[d] - 2)
                mid = 0.5 * (k + other) * h[d]
                xs = [x0, x1]
                xs[d] = mid
                slope = c[d] + 2 * c[2 + d] * mid + c[4] * xs[1 - d]
                assert abs(fd - slope) < 1e-12
            assert abs(adr.tau1_second_derivative(g, tau1, i, d) - d2[d]) < 1e-10


def test_tau0_derivatives_identities():
    g = adr.Grid((7, 6, 5), (0.3, 0.2, 0.1))
    src = (2, 1, 3)
    for j in range(g.N):
        i = g.coords(j)
        r, d1, d2 = adr.tau0_derivatives(g, src, i)
        if r == 0:
            continue
        assert abs(sum(v * v for v in d1) - 1.0) < 1e-14          # |grad tau0| = 1
        assert abs(sum(d2) - 2.0 / r) < 1e-12 * (1 + 2.0 / r)      # Delta tau0 = (d - 1)/r
        # finite-difference check of the analytic derivatives
        eps = 1e-6
        for d in range(3):
            xp = [(i[k] - src[k]) * g.h[k] for k in range(3)]
            xm = list(xp)
            xp[d] += eps
            xm[d] -= eps
            fd = (math.dist(xp, [0, 0, 0]) - math.dist(xm, [0, 0, 0])) / (2 * eps)
            assert abs(fd - d1[d]) < 1e-7


def test_constant_medium_reaction_vanishes():
    """Exact eikonal in a constant medium: w^2 (kappa^2 - |grad tau|^2) = 0 (Eq. eikonal)."""
    P = W.constant_medium((17, 13), kappa0=0.8)
    g = adr.Grid(P.n, P.h)
    for j in range(0, g.N, 7):
        if g.coords(j) == P.src:
            continue
        _, gr, t, rho = adr.node_coefficients(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, j)
        assert abs(rho.real) < 1e-9 * P.omega ** 2
        r = adr.tau0_derivatives(g, P.src, g.coords(j))[0]
        assert abs(sum(t) - 0.8 / r) < 1e-9 / r          # Delta tau = kappa (d-1)/r in 2D


def test_reconstruct_phase():
    P = W.constant_medium((9, 9), kappa0=1.0)
    g = adr.Grid(P.n, P.h)
    a = np.arange(g.N) + 1j
    u = adr.reconstruct(g, P.src, P.omega, P.tau1, a)
    tau = adr.travel_time(g, P.src, P.tau1)
    assert np.allclose(np.abs(u), np.abs(a), rtol=0, atol=1e-12)
    assert np.allclose(u * np.exp(1j * P.omega * tau), a, rtol=1e-14, atol=1e-12)


def test_shifted_laplacian_preconditioner():
    """Eq. shift: with tau = 0 the preconditioner is the Helmholtz matrix of
    Eq. HelmholtzLinSystem minus i alpha w^2 kappa^2 on the diagonal; alpha = 0
    gives the unshifted operator; the shift moves every Rayleigh quotient down
    in the complex plane by alpha w^2 <kappa^2> (the damping that makes the
    multigrid cycle work, Sec. 3)."""
    P = W.marine_2d((17, 17))
    g = adr.Grid(P.n, P.h)
    tau1 = np.zeros(g.N)
    H = adr.assemble_helmholtz(g, P.omega, P.kappa, P.gamma)
    A0 = adr.assemble_preconditioner(g, P.src, P.omega, P.kappa, P.gamma, tau1)
    A5 = adr.assemble_preconditioner(g, P.src, P.omega, P.kappa, P.gamma, tau1, shift=0.5)
    assert abs(A0 - H).max() <= 1e-12 * abs(H).max()
    D = (A5 - H).tocsr()
    assert D.nnz == g.N and np.allclose(D.diagonal(), -0.5j * P.omega ** 2 * P.kappa ** 2, rtol=1e-14, atol=0)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(g.N) + 1j * rng.standard_normal(g.N)
    q0 = np.vdot(x, A0 @ x) / np.vdot(x, x)
    q5 = np.vdot(x, A5 @ x) / np.vdot(x, x)
    expect = 0.5 * P.omega ** 2 * np.vdot(x, P.kappa ** 2 * x).real / np.vdot(x, x).real
    assert abs((q0 - q5).imag - expect) <= 1e-10 * expect and abs((q0 - q5).real) <= 1e-10 * abs(q0)
