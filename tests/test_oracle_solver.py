"""Pins of the oracle's multigrid, Krylov and fast-marching code, and of the
whole discretisation against closed-form solutions (no GPU).

* P reproduces (multi)linear functions exactly; the Galerkin product of the
  constant-coefficient Laplacian has the known interior stencil
  (Eq. coarseGridMatrix with bilinear P: 1D [1/2, -1, 1/2] / h^2, 2D its
  tensor combination with P^T P = [1/4, 3/2, 1/4]);
* GMRES with as many steps as unknowns is a direct solve; one Jacobi-GMRES
  step is the minimal-residual relaxation; FGMRES agrees with a sparse
  direct solve;
* the fast-marching travel time is exact in a constant medium and converges
  to the textbook travel time of a linear velocity gradient;
* the ADR solution converges to the free-space Hankel amplitude and the
  standard discretisation's phase error shows where the ADR form wins
  (Sec. 4.1, linear model).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.special as ss

from oracle import adr, eikonal, krylov
from oracle import multigrid as mg
from paper_1712_06091_gb300 import workloads as W


def test_prolongation_exact_on_linear_functions():
    n = (9, 7, 5)
    P = mg.prolongation(n)
    nc = mg.coarse_shape(n)
    Xf = W.node_coordinates(n, (1.0, 1.0, 1.0))
    Xc = W.node_coordinates(nc, (2.0, 2.0, 2.0))
    for f in (lambda x: 1.0 + 0 * x[0], lambda x: x[0], lambda x: x[1] - 2 * x[2], lambda x: x[0] * x[1] * x[2]):
        assert np.allclose(P @ f(Xc), f(Xf), atol=1e-12)


def test_galerkin_laplacian_closed_form():
    # 1D: P^T L_h P = [1/2, -1, 1/2] / h^2 in the interior
    nf = 17
    h = 0.1
    L1 = sp.diags([np.ones(nf - 1), -2 * np.ones(nf), np.ones(nf - 1)], [-1, 0, 1]) / h ** 2
    P1 = mg.interpolation_1d(nf)
    Lc = (P1.T @ L1 @ P1).toarray()
    i = 4
    assert np.allclose(Lc[i, i - 1:i + 2], np.array([0.5, -1.0, 0.5]) / h ** 2)
    assert np.allclose(Lc[i, :i - 1], 0) and np.allclose(Lc[i, i + 2:], 0)
    # 2D: (P^T L_x P) (x) (P^T P)_y + (P^T P)_x (x) (P^T L_y P)
    n = (17, 13)
    hx, hy = 0.1, 0.25
    g = adr.Grid(n, (hx, hy))
    H = adr.assemble_helmholtz(g, 1e-30, np.zeros(g.N), np.zeros(g.N))   # the Laplacian with Neumann rows
    P = mg.prolongation(n)
    Ac = (P.T @ H @ P).tocsr()
    nc = mg.coarse_shape(n)
    gc = adr.Grid(nc, (2 * hx, 2 * hy))
    I = gc.index((4, 3))
    lap = np.array([0.5, -1.0, 0.5])
    ptp = np.array([0.25, 1.5, 0.25])
    expect = np.outer(ptp, lap) / hx ** 2 + np.outer(lap, ptp) / hy ** 2   # [dy, dx]
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            J = gc.index((4 + dx, 3 + dy))
            assert abs(Ac[I, J] - expect[dy + 1, dx + 1]) < 1e-9 * np.abs(expect).max()
    assert Ac[I].nnz == 9


def _small_system(seed=0, n=(9, 7)):
    P = W.constant_medium(n, kappa0=1.0, ppw=6)
    g = adr.Grid(P.n, P.h)
    A = adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, "2up")
    b = W.random_complex(g.N, seed)
    return g, P, A, b


def test_coarse_gmres_full_dimension_is_direct_solve():
    g, P, A, b = _small_system(n=(5, 5))
    dinv = 1.0 / A.diagonal()
    x = mg.coarse_gmres(A, dinv, b, g.N)
    xe = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xe) <= 1e-9 * np.linalg.norm(xe)


def test_mr_relaxation_is_one_gmres_step():
    g, P, A, b = _small_system()
    dinv = 1.0 / A.diagonal()
    x = W.random_complex(g.N, 3)
    got = mg.relax_mr(A, dinv, x, b)
    ref = x + mg.coarse_gmres(A, dinv, b - A @ x, 1)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_fgmres_matches_direct_solve_and_is_monotone():
    P = W.constant_medium((33, 33))
    g = adr.Grid(P.n, P.h)
    A = adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, "2up")
    Ap = adr.assemble_preconditioner(g, P.src, P.omega, P.kappa, P.gamma, P.tau1)
    hier = mg.build_hierarchy(Ap, P.n, 3)
    q = adr.point_source_rhs(g, P.src)
    prm = mg.CycleParams()
    x, its, rel, hist = krylov.fgmres(A, q, lambda v: mg.cycle(hier, v, prm), tol=1e-12, restart=8, maxit=200)
    xe = spla.spsolve(A.tocsc(), q)
    assert rel <= 1e-12
    assert np.linalg.norm(x - xe) <= 1e-10 * np.linalg.norm(xe)
    # GMRES minimises the residual over a growing space within each cycle
    for c in range(0, len(hist), 8):
        seg = hist[c:c + 8]
        assert all(seg[k + 1] <= seg[k] * (1 + 1e-12) for k in range(len(seg) - 1))
    # explicit residual agrees with the definition
    assert abs(np.linalg.norm(q - A @ x) / np.linalg.norm(q) - rel) < 1e-14


def test_selective_gram_schmidt_reorthogonalises_only_on_cancellation():
    rng = np.random.default_rng(5)
    n, k = 400, 12
    V, _ = np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))
    # mild cancellation: one pass, exact decomposition w = V h + w'
    w = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    h, w1 = krylov.cgs_selective(V, w, 0.1)
    assert np.linalg.norm(w - (V @ h + w1)) <= 1e-14 * np.linalg.norm(w)
    h_one = V.conj().T @ w
    assert np.array_equal(h, h_one)                      # no second pass taken
    assert np.linalg.norm(V.conj().T @ w1) <= 1e-14 * np.linalg.norm(w1)
    # severe cancellation (|w'| = 1e-8 |w|): one pass leaves V-components of
    # relative size ~eps/1e-8; the test triggers the second pass, which removes them
    c = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    u -= V @ (V.conj().T @ u)
    w = V @ c + 1e-8 * np.linalg.norm(c) * u / np.linalg.norm(u)
    _, w_single = krylov.cgs_selective(V, w, 0.0)
    h, w_sel = krylov.cgs_selective(V, w, 0.1)
    loss = lambda x: np.linalg.norm(V.conj().T @ x) / np.linalg.norm(x)
    assert loss(w_single) > 1e-12
    assert loss(w_sel) < 1e-14
    assert np.linalg.norm(h - c) <= 1e-12 * np.linalg.norm(c)


def test_fgmres_selective_reorthogonalisation_matches_cgs2():
    P = W.constant_medium((33, 33))
    g = adr.Grid(P.n, P.h)
    A = adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, "2up")
    Ap = adr.assemble_preconditioner(g, P.src, P.omega, P.kappa, P.gamma, P.tau1)
    hier = mg.build_hierarchy(Ap, P.n, 3)
    q = adr.point_source_rhs(g, P.src)
    prm = mg.CycleParams()
    pc = lambda v: mg.cycle(hier, v, prm)
    x2, its2, rel2, _ = krylov.fgmres(A, q, pc, tol=1e-12, restart=8, maxit=200)
    xs, itss, rels, _ = krylov.fgmres(A, q, pc, tol=1e-12, restart=8, maxit=200, reorth_eta=0.1)
    assert rels <= 1e-12 and abs(itss - its2) <= 1
    assert np.linalg.norm(xs - x2) <= 1e-10 * np.linalg.norm(x2)


def test_kcycle_fgmres_inner_is_fixed_count():
    g, P, A, b = _small_system(n=(17, 17))
    Ap = adr.assemble_preconditioner(adr.Grid(P.n, P.h), P.src, P.omega, P.kappa, P.gamma, P.tau1)
    hier = mg.build_hierarchy(Ap, P.n, 3)
    prm = mg.CycleParams(cycle="K", kcycle_iterations=2)
    z1 = mg.cycle(hier, b, prm)
    z2 = mg.cycle(hier, 2.0 * b, prm)
    assert np.allclose(z2, 2.0 * z1, rtol=1e-12, atol=0)   # scale invariance of the nonlinear cycle


def test_vcycle_poisson_contraction():
    """Textbook V(1,1) damped-Jacobi behaviour on a shifted Neumann Laplacian (SPD)."""
    n = (65, 65)
    g = adr.Grid(n, (1 / 64, 1 / 64))
    Lap = adr.assemble_helmholtz(g, 1e-30, np.zeros(g.N), np.zeros(g.N))
    A = (-Lap + sp.identity(g.N) * 1.0).tocsr()
    hier = mg.build_hierarchy(A, n, 5)
    prm = mg.CycleParams(cycle="V", relax="jacobi", pre=[1] * 8, post=[1] * 8, weights=[0.8] * 8,
                         coarse_iterations=30)
    b = np.zeros(g.N, dtype=np.complex128)
    x = W.random_complex(g.N, 1)
    r0 = np.linalg.norm(b - A @ x)
    for _ in range(8):
        x = x + mg.cycle(hier, b - A @ x, prm)
    factor = (np.linalg.norm(b - A @ x) / r0) ** (1 / 8)
    assert factor < 0.35, factor


def test_fast_marching_constant_medium_exact():
    for n, src in (((21, 13), (3, 0)), ((9, 8, 7), (4, 0, 3))):
        g = adr.Grid(n, tuple(0.1 * (d + 1) for d in range(len(n))))
        for order in (1, 2):
            t1 = eikonal.factored_fast_marching(g, np.full(g.N, 0.6), src, order)
            assert np.abs(t1 - 0.6).max() < 1e-12


def test_fast_marching_linear_gradient_convergence():
    errs = {1: [], 2: []}
    for n in (33, 65, 129):
        nn = (n, (n + 1) // 2)
        src = ((nn[0] - 1) // 2, 2)
        P = W.linear_velocity(nn, (2.0, 1.0), 1.5, 1.0, src)
        g = adr.Grid(P.n, P.h)
        ref = W.linear_velocity_traveltime(P.n, P.h, src, 1.5, 1.0)
        tau0 = adr.travel_time(g, src, np.ones(g.N))
        for order in (1, 2):
            t1 = eikonal.factored_fast_marching(g, P.kappa, src, order)
            errs[order].append(np.abs((t1 - ref) * tau0).max())
    r1 = [math.log2(errs[1][k] / errs[1][k + 1]) for k in range(2)]
    r2 = [math.log2(errs[2][k] / errs[2][k + 1]) for k in range(2)]
    assert min(r1) > 0.75, (errs, r1)
    assert min(r2) > 1.6, (errs, r2)
    assert errs[2][-1] < errs[1][-1] / 4


def _amplitude_error_2d(n, scheme, near_radius):
    """Median relative error of the ADR amplitude against the free-space amplitude
    (i/4) H0^(2)(w r) e^{i w r} on 0.1 < r < 0.35 (source at the centre of a 2 x 2
    domain, wavelength 0.2, absorbing layers three wavelengths thick so that the
    wall reflection, attenuated by about exp(-2 pi), stays below the errors measured)."""
    extent, lam = 2.0, 0.2
    omega = 2 * math.pi / lam
    P = W.constant_medium((n, n), extent=extent)
    h = P.h[0]
    gamma, _ = W.absorbing_layer(P.n, P.h, P.kappa, omega, W.all_faces(2), widths=[int(round(3 * lam / h))] * 4)
    g = adr.Grid(P.n, P.h)
    q = adr.point_source_rhs(g, P.src)
    X = W.node_coordinates(P.n, P.h)
    r = np.sqrt((X[0] - 1.0) ** 2 + (X[1] - 1.0) ** 2)
    mask = (r > 0.1) & (r < 0.35)
    ref = 0.25j * ss.hankel2(0, omega * r[mask]) * np.exp(1j * omega * r[mask])
    if scheme == "std":
        u = spla.spsolve(adr.assemble_helmholtz(g, omega, P.kappa, gamma).tocsc(), q)
        a = u[mask] * np.exp(1j * omega * r[mask])
    else:
        A = adr.assemble_adr(g, P.src, omega, P.kappa, gamma, P.tau1, scheme, near_radius)
        a = spla.spsolve(A.tocsc(), q)[mask]
    return float(np.median(np.abs(a - ref) / np.abs(ref)))


def test_adr_amplitude_matches_hankel_and_converges():
    """Sec. 1 closed form (2D via the Hankel function) at fixed omega, h -> h/2.

    With central advection within two nodes of the source the upwind ADR
    amplitude converges at second order; with the literal one-node
    neighbourhood a bounded, h-independent amplitude bias of a few percent
    remains (the second-order upwind rows two nodes away reach into the
    singular source node).  The standard scheme at 12.8 points per wavelength
    carries the dispersion error that the ADR form avoids (Sec. 4.1)."""
    e1 = _amplitude_error_2d(129, "2up", 2)
    e2 = _amplitude_error_2d(257, "2up", 2)
    assert e2 < 0.03 and e2 < e1 / 3.0, (e1, e2)
    b1 = _amplitude_error_2d(129, "2up", 1)
    b2 = _amplitude_error_2d(257, "2up", 1)
    assert 0.03 < b2 < 0.09 and abs(b2 - b1) < 0.01, (b1, b2)
    s1 = _amplitude_error_2d(129, "std", 1)
    assert s1 > 0.05, s1
