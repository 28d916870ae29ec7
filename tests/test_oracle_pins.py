"""Further pins of the oracle against what the paper and the mathematics fix
(no GPU):

* the reconstruction u = a exp(-i w tau) (Eq. new_u) of the upwind ADR
  solution satisfies the standard 5-point Helmholtz discretisation
  (Eq. HelmholtzLinSystem) away from the source with a residual that falls as
  O(h^2) at fixed omega (Eq. matrix_rescaling: the ADR rows are M^{-1} H M up
  to O(h^2)); the same field with the opposite phase does not;
* the 3D constant-medium amplitude converges to the closed form
  a = -1/(4 pi r) of Sec. 1 (q = +delta, u = -exp(-i w kappa r)/(4 pi r));
* the Krylov cycle (Alg. Kcycle) with an exact inner solve equals the
  two-grid cycle of Alg. TwoGrid written out with dense matrices: relaxation,
  residual restriction by P^T, exact coarse solve, prolongation, relaxation.
"""
import math

import numpy as np
import scipy.sparse.linalg as spla

from oracle import adr, krylov
from oracle import multigrid as mg
from paper_1712_06091_gb300 import workloads as W

# ---------------------------------------------------------------------------
# Reconstruction: Helmholtz residual of u = a exp(-i w tau)
# ---------------------------------------------------------------------------
FREQ = 4.0            # wavelength 0.25 on a 2 x 2 square
EXTENT = 2.0
LAYER_WAVELENGTHS = 3  # thick enough that the layer's reflection stays below the O(h^2) term


def _reconstruction_residual(n, phase_sign=-1, plain=False):
    """Relative 5-point Helmholtz residual of the reconstructed ADR solution on
    the nodes farther than 0.1 from the source and outside the layer (2D
    constant medium, fixed omega).  phase_sign = +1 replaces the phase of
    Eq. new_u by its conjugate (a planted sign error)."""
    omega = 2.0 * math.pi * FREQ
    P = W.constant_medium((n, n), extent=EXTENT)
    cells = int(round(LAYER_WAVELENGTHS / FREQ / P.h[0]))
    gamma, _ = W.absorbing_layer(P.n, P.h, P.kappa, omega, W.all_faces(2), widths=[cells] * 4)
    g = adr.Grid(P.n, P.h)
    tau1 = adr.PlainTau(adr.travel_time(g, P.src, P.tau1)) if plain else P.tau1
    A = adr.assemble_adr(g, P.src, omega, P.kappa, gamma, tau1, "2up")
    q = adr.point_source_rhs(g, P.src)
    a = spla.spsolve(A.tocsc(), q)
    if phase_sign < 0:
        u = adr.reconstruct(g, P.src, omega, tau1, a)
    else:
        u = a * np.exp(+1j * omega * adr.travel_time(g, P.src, tau1))
    res = adr.assemble_helmholtz(g, omega, P.kappa, gamma) @ u - q
    X = W.node_coordinates(P.n, P.h)
    r = np.sqrt(sum((x - s * hh) ** 2 for x, s, hh in zip(X, P.src, P.h)))
    far = (r > 0.1) & (gamma == 0.0)
    scale = omega ** 2 * P.kappa[far] ** 2 * np.abs(u[far])     # size of the reaction term
    return float(np.linalg.norm(res[far]) / np.linalg.norm(scale))


def test_reconstruction_satisfies_helmholtz_to_second_order():
    """Eq. new_u with Eq. matrix_rescaling: H (M a) = M (M^{-1} H M) a, and
    M^{-1} H M differs from the upwind ADR matrix by O(h^2) on smooth a, so the
    reconstructed field solves the 5-point Helmholtz system away from the
    source up to O(h^2).  Measured: 4.9e-2, 1.0e-2, 2.5e-3 (rates 2.3, 2.0).
    The conjugate phase exp(+i w tau) turns the outgoing wave into an incoming
    one, which solves the homogeneous equation only asymptotically: its
    residual stalls (measured 3.3e-2 at 257^2) instead of converging."""
    e = [_reconstruction_residual(n) for n in (65, 129, 257)]
    rates = [math.log2(e[k] / e[k + 1]) for k in range(2)]
    assert min(rates) > 1.8, (e, rates)
    assert e[-1] < 4e-3, e
    wrong = [_reconstruction_residual(n, phase_sign=+1) for n in (129, 257)]
    assert wrong[1] > 0.5 * wrong[0] and wrong[1] > 8 * e[-1], (wrong, e)


# ---------------------------------------------------------------------------
# 3D closed form a = -1/(4 pi r)
# ---------------------------------------------------------------------------
def _amplitude_error_3d(n, near_radius):
    """Median relative error of the 3D ADR amplitude against -1/(4 pi r) on the
    nodes at least five cells from the source and outside the layer (constant
    medium on a cube of four wavelengths, layer one wavelength thick on every
    face, fixed omega).  Returns (median error, median of a * (-4 pi r))."""
    freq, extent = 1.0, 4.0
    omega = 2.0 * math.pi * freq
    P = W.constant_medium((n, n, n), extent=extent)
    cells = int(round(1.0 / freq / P.h[0]))
    gamma, _ = W.absorbing_layer(P.n, P.h, P.kappa, omega, W.all_faces(3), widths=[cells] * 6)
    g = adr.Grid(P.n, P.h)
    A2 = adr.assemble_adr(g, P.src, omega, P.kappa, gamma, P.tau1, "2up", near_radius)
    A1 = adr.assemble_adr(g, P.src, omega, P.kappa, gamma, P.tau1, "1up", near_radius)
    hier = mg.build_hierarchy((0.75 * A2 + 0.25 * A1).tocsr(), P.n, 3)    # Eq. precADRup
    q = adr.point_source_rhs(g, P.src)
    a, _, rel, _ = krylov.fgmres(A2, q, lambda v: mg.cycle(hier, v, mg.CycleParams()), tol=1e-9, restart=20,
                                 maxit=300)
    assert rel <= 1e-9
    X = W.node_coordinates(P.n, P.h)
    r = np.sqrt(sum((x - s * hh) ** 2 for x, s, hh in zip(X, P.src, P.h)))
    far = (r >= 5 * P.h[0]) & (gamma == 0.0)
    ref = -1.0 / (4.0 * math.pi * r[far])
    return (float(np.median(np.abs(a[far] - ref) / np.abs(ref))),
            complex(np.median((a[far] / ref).real) + 1j * np.median((a[far] / ref).imag)))


def test_3d_amplitude_converges_to_closed_form():
    """Sec. 1: in a constant medium the 3D Green's function is
    -exp(-i w kappa r)/(4 pi r), so the amplitude is -1/(4 pi r) for every
    omega.  With central advection within two nodes of the source the error
    falls at (at least) second order from 8 to 12 points per wavelength
    (measured 0.295 -> 0.109); the sign and size are fixed by the ratio
    a / (-1/(4 pi r)) staying near +1."""
    e8, ratio8 = _amplitude_error_3d(33, 2)
    e12, ratio12 = _amplitude_error_3d(49, 2)
    assert e12 < 0.15 and e8 / e12 > (49 - 1) ** 2 / (33 - 1) ** 2 * 0.9, (e8, e12)
    assert abs(ratio12 - 1.0) < 0.2, ratio12


# ---------------------------------------------------------------------------
# Alg. Kcycle against the explicit two-grid formula of Alg. TwoGrid
# ---------------------------------------------------------------------------
def _dense_interpolation(nf):
    """Linear interpolation from every other node: weights 1 on coinciding
    nodes, 1/2 on the two coarse neighbours of a fine node between them."""
    nc = (nf - 1) // 2 + 1
    P = np.zeros((nf, nc))
    for i in range(nf):
        if i % 2 == 0:
            P[i, i // 2] = 1.0
        else:
            P[i, i // 2] = P[i, i // 2 + 1] = 0.5
    return P


def _jacobi_dense(A, x, b, w, sweeps):
    d = np.diag(A)
    for _ in range(sweeps):
        x = x + w * (b - A @ x) / d
    return x


def test_kcycle_with_exact_inner_solve_is_the_two_grid_cycle():
    """With kcycle_iterations equal to the level-1 dimension the inner FGMRES
    of Alg. Kcycle solves A_1 e = r_1 exactly, and the coarsest GMRES with as
    many steps as unknowns is exact too, so a 3-level K-cycle must equal the
    two-grid cycle of Alg. TwoGrid on level 0 with an exact coarse solve:
        x1 = nu1 Jacobi sweeps from 0,
        x2 = x1 + P A_1^{-1} P^T (b - A x1),   A_1 = P^T A P,
        x3 = nu2 Jacobi sweeps from x2.
    A mistake in the recursion (restricting b instead of b - A x, a dropped
    post-relaxation, the inner solve on the wrong level, P^T / P swapped)
    changes x3."""
    P0 = W.marine_2d((9, 9))
    g = adr.Grid(P0.n, P0.h)
    A = adr.assemble_preconditioner(g, P0.src, P0.omega, P0.kappa, P0.gamma,
                                    W.smooth_random_field(P0.n, seed=2) * P0.kappa.mean())
    hier = mg.build_hierarchy(A, P0.n, 3)
    assert [lv["n"] for lv in hier] == [(9, 9), (5, 5), (3, 3)]
    b = W.random_complex(g.N, 7)
    nu1, nu2, w = 2, 3, 0.6
    prm = mg.CycleParams(cycle="K", relax="jacobi", pre=[nu1] * 8, post=[nu2] * 8, weights=[w] * 8,
                         coarse_iterations=9, kcycle_iterations=25)
    got = mg.cycle(hier, b, prm)

    Ad = A.toarray()
    Pd = np.kron(_dense_interpolation(9), _dense_interpolation(9))     # axis 0 fastest
    A1 = Pd.T @ Ad @ Pd
    x1 = _jacobi_dense(Ad, np.zeros(g.N, dtype=complex), b, w, nu1)
    x2 = x1 + Pd @ np.linalg.solve(A1, Pd.T @ (b - Ad @ x1))
    x3 = _jacobi_dense(Ad, x2, b, w, nu2)
    assert np.linalg.norm(got - x3) <= 1e-9 * np.linalg.norm(x3), np.linalg.norm(got - x3) / np.linalg.norm(x3)
    # the V-cycle with the same settings is not exact on level 1, so it differs
    v = mg.cycle(hier, b, mg.CycleParams(cycle="V", relax="jacobi", pre=[nu1] * 8, post=[nu2] * 8, weights=[w] * 8,
                                         coarse_iterations=9))
    assert np.linalg.norm(v - x3) > 1e-6 * np.linalg.norm(x3)


def test_kcycle_one_inner_step_is_a_minimal_residual_scaling():
    """Alg. Kcycle with FGMRES(1) on level 1: e_1 = alpha c with c the cycle
    applied to the restricted residual r_1 and alpha = (A_1 c)^H r_1 /
    |A_1 c|^2, the one-dimensional least-squares solution; everything else is
    the V-cycle's."""
    P0 = W.marine_2d((17, 17))
    g = adr.Grid(P0.n, P0.h)
    A = adr.assemble_preconditioner(g, P0.src, P0.omega, P0.kappa, P0.gamma, P0.kappa.copy())
    hier = mg.build_hierarchy(A, P0.n, 3)
    b = W.random_complex(g.N, 8)
    kw = dict(relax="jacobi", pre=[1] * 8, post=[1] * 8, weights=[0.7] * 8, coarse_iterations=6)
    got = mg.cycle(hier, b, mg.CycleParams(cycle="K", kcycle_iterations=1, **kw))
    vprm = mg.CycleParams(cycle="V", **kw)
    lv = hier[0]
    x1 = mg.jacobi(lv["A"], lv["dinv"], np.zeros_like(b), b, 0.7)
    r1 = lv["P"].T @ (b - lv["A"] @ x1)
    c = mg.cycle(hier, r1, vprm, level=1)
    Ac = hier[1]["A"] @ c
    alpha = np.vdot(Ac, r1) / np.vdot(Ac, Ac).real
    x2 = x1 + lv["P"] @ (alpha * c)
    x3 = mg.jacobi(lv["A"], lv["dinv"], x2, b, 0.7)
    assert np.linalg.norm(got - x3) <= 1e-12 * np.linalg.norm(x3)


# ---------------------------------------------------------------------------
# Alg. Kcycle's early exit (the 0.1 coarse threshold of Sec. 4.2)
# ---------------------------------------------------------------------------
def _level1_system():
    P0 = W.marine_2d((33, 33))
    g = adr.Grid(P0.n, P0.h)
    A = adr.assemble_preconditioner(g, P0.src, P0.omega, P0.kappa, P0.gamma, P0.kappa.copy())
    hier = mg.build_hierarchy(A, P0.n, 4)
    prm = mg.CycleParams(cycle="K")
    b = W.random_complex(hier[1]["A"].shape[0], 9)
    return hier, prm, b


def test_kcycle_inner_solve_threshold_semantics():
    """The inner FGMRES stops after the first step exactly when that step's
    residual |b - A x_1| (x_1 = alpha z_0, the one-dimensional least-squares
    solution along z_0 = B(b/|b|)) is at most threshold |b|; threshold 0 is the
    fixed-count inner solve."""
    hier, prm, b = _level1_system()
    A1 = hier[1]["A"]
    pc = lambda v: mg.cycle(hier, v, prm, level=1)
    fixed = mg.fixed_fgmres(A1, b, pc, 2)
    x0, k0 = mg.kcycle_fgmres(A1, b, pc, 2, 0.0)
    assert k0 == 2 and np.linalg.norm(x0 - fixed) <= 1e-13 * np.linalg.norm(fixed)
    z0 = pc(b / np.linalg.norm(b))
    Az = A1 @ z0
    alpha = np.vdot(Az, b) / np.vdot(Az, Az).real
    ratio = np.linalg.norm(b - alpha * Az) / np.linalg.norm(b)
    assert 0.0 < ratio < 1.0
    x_hi, k_hi = mg.kcycle_fgmres(A1, b, pc, 2, ratio * (1 + 1e-9))
    x_lo, k_lo = mg.kcycle_fgmres(A1, b, pc, 2, ratio * (1 - 1e-9))
    assert k_hi == 1 and k_lo == 2
    assert np.linalg.norm(x_hi - alpha * z0) <= 1e-12 * np.linalg.norm(alpha * z0)
    assert np.linalg.norm(x_lo - fixed) <= 1e-13 * np.linalg.norm(fixed)


def test_kcycle_threshold_one_is_the_one_step_kcycle():
    """With a threshold of 1 the first step always satisfies it (a least-squares
    step never increases the residual), so the cycle is the K-cycle with
    FGMRES(1), pinned above by the minimal-residual scaling."""
    P0 = W.marine_2d((33, 33))
    g = adr.Grid(P0.n, P0.h)
    A = adr.assemble_preconditioner(g, P0.src, P0.omega, P0.kappa, P0.gamma, P0.kappa.copy())
    hier = mg.build_hierarchy(A, P0.n, 4)
    b = W.random_complex(g.N, 10)
    one = mg.cycle(hier, b, mg.CycleParams(cycle="K", kcycle_iterations=1))
    thr = mg.cycle(hier, b, mg.CycleParams(cycle="K", kcycle_iterations=2, kcycle_threshold=1.0))
    assert np.linalg.norm(thr - one) <= 1e-13 * np.linalg.norm(one)


# ---------------------------------------------------------------------------
# Plain travel time (finite-difference coefficients)
# ---------------------------------------------------------------------------
def test_plain_tau_coefficients_exact_on_a_plane_wave():
    """For a linear tau (a plane wave, tau = k.x + c) every difference rule is
    exact: grad tau = k, d_dd tau = 0 and the reaction is
    w^2 (kappa^2 - |k|^2) - i w gamma kappa^2 at every node, boundary included."""
    n, h = (9, 7, 6), (0.1, 0.15, 0.2)
    g = adr.Grid(n, h)
    X = W.node_coordinates(n, h)
    k = (0.3, -0.5, 0.4)
    tau = 0.7 + sum(kd * x for kd, x in zip(k, X))
    kappa = W.smooth_random_field(n, seed=3)
    gamma = np.linspace(0.0, 2.0, g.N)
    omega = 5.0
    for j in range(g.N):
        tv, gr, t, rho = adr.node_coefficients(g, (4, 3, 2), omega, kappa, gamma, adr.PlainTau(tau), j)
        assert tv == tau[j]
        assert max(abs(a - b) for a, b in zip(gr, k)) < 1e-12
        assert max(abs(v) for v in t) < 1e-9
        k2 = kappa[j] ** 2
        assert abs(rho - (omega ** 2 * (k2 - sum(v * v for v in k)) - 1j * omega * gamma[j] * k2)) < 1e-9


def test_plain_tau_converges_to_factored_coefficients():
    """tau = kappa r sampled on the grid: away from the source the differences
    of tau converge to the analytic derivatives of Eq. travel_time_coeff at
    second order (measured at a fixed physical point); at the source's
    neighbours they do not (the conical kink), which is why the factored form
    is the accurate input."""
    errs = []
    for n in (17, 33, 65):
        P = W.constant_medium((n, n), kappa0=0.8)
        g = adr.Grid(P.n, P.h)
        tau = adr.travel_time(g, P.src, P.tau1)
        c = (n - 1) // 2
        j = g.index((c + (n - 1) // 4, c + (n - 1) // 8))      # physical offset (0.25, 0.125)
        _, gf, tf, _ = adr.node_coefficients(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, j)
        _, gp, tp, _ = adr.node_coefficients(g, P.src, P.omega, P.kappa, P.gamma, adr.PlainTau(tau), j)
        errs.append(max(abs(a - b) for a, b in zip(gf + tf, gp + tp)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 1.8, (errs, rates)
    # at the diagonal neighbour of the source the central difference spans the
    # kink: kappa (sqrt 5 - 1) / 2 against the analytic kappa / sqrt 2, at any h
    for n in (33, 65):
        P = W.constant_medium((n, n), kappa0=0.8)
        g = adr.Grid(P.n, P.h)
        tau = adr.travel_time(g, P.src, P.tau1)
        j = g.index((P.src[0] + 1, P.src[1] + 1))
        _, gf, _, _ = adr.node_coefficients(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, j)
        _, gp, _, _ = adr.node_coefficients(g, P.src, P.omega, P.kappa, P.gamma, adr.PlainTau(tau), j)
        assert abs(gf[0] - 0.8 / math.sqrt(2)) < 1e-12 and abs(gp[0] - 0.4 * (math.sqrt(5) - 1)) < 1e-12


def test_plain_tau_reconstruction_satisfies_helmholtz_to_second_order():
    """The same Helmholtz-residual pin for the plain-tau coefficients (tau = kappa r
    given as values): away from the source the finite differences of tau are
    second-order accurate, so the reconstructed field again solves the 5-point
    system to O(h^2) (measured 4.7e-2, 7.7e-3, 1.9e-3)."""
    e = [_reconstruction_residual(n, plain=True) for n in (65, 129, 257)]
    rates = [math.log2(e[k] / e[k + 1]) for k in range(2)]
    assert min(rates) > 1.8 and e[-1] < 4e-3, (e, rates)


def test_selective_coarse_gmres():
    """The coarsest GMRES with the selective second Gram-Schmidt pass (reading
    M2): with as many steps as unknowns it is still a direct solve, and on a
    coarse Galerkin operator, where the first pass never cancels much, it
    equals the classical-twice iteration up to rounding."""
    g, P, A, b = None, None, None, None
    P0 = W.constant_medium((5, 5), kappa0=1.0, ppw=6)
    g = adr.Grid(P0.n, P0.h)
    A = adr.assemble_adr(g, P0.src, P0.omega, P0.kappa, P0.gamma, P0.tau1, "2up")
    b = W.random_complex(g.N, 4)
    dinv = 1.0 / A.diagonal()
    xe = spla.spsolve(A.tocsc(), b)
    x = mg.coarse_gmres(A, dinv, b, g.N, reorth_eta=0.1)
    assert np.linalg.norm(x - xe) <= 1e-9 * np.linalg.norm(xe)
    M = W.marine_2d((65, 65))
    gm = adr.Grid(M.n, M.h)
    Ap = adr.assemble_preconditioner(gm, M.src, M.omega, M.kappa, M.gamma, M.kappa.copy())
    hier = mg.build_hierarchy(Ap, M.n, 3)
    c = hier[-1]
    r = W.random_complex(c["A"].shape[0], 5)
    x2 = mg.coarse_gmres(c["A"], c["dinv"], r, 10)
    xs = mg.coarse_gmres(c["A"], c["dinv"], r, 10, reorth_eta=0.1)
    assert np.linalg.norm(xs - x2) <= 1e-13 * np.linalg.norm(x2)
