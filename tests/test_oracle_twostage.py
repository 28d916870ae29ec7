"""Pins of the oracle's two-stage central solve (Algorithm ADRlong), no GPU.

* the rescaled central matrix M H_cen M^{-1} has, at the source, exactly the
  standard Helmholtz row (the source row of H_hat is the row of M^{-1} H M,
  Eq. helmADR2), which fixes the direction of the rescaling;
* with tau = 0 the stage-2 preconditioner H_s^cen is the shifted-Laplacian
  matrix H - i alpha w^2 diag(kappa^2) of Eq. shift;
* the result solves H_cen a = q_hat (compared with a sparse direct solve), and
  u = M a solves the rescaled system with the same relative residual (M is
  unitary);
* stage 1 stops by its rule (at most 5 iterations or residual 1e-2 of Eq. 1up).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import adr, eikonal, krylov, twostage
from oracle import multigrid as mg
from paper_1712_06091_gb300 import workloads as W

PRM = mg.CycleParams(cycle="K", relax="mr", pre=[2, 3, 4], post=[2, 3, 4], weights=[0.5] * 3, coarse_iterations=10,
                     kcycle_iterations=2)


def _marine(n=(33, 33)):
    P = W.marine_2d(n)
    g = adr.Grid(P.n, P.h)
    P.tau1 = eikonal.factored_fast_marching(g, P.kappa, P.src, order=2)
    return P, g


def test_rescaled_central_source_row_is_helmholtz():
    P, g = _marine()
    m = twostage.phase(g, P.src, P.omega, P.tau1)
    Ar = twostage.rescaled(adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, "cen"), m)
    H = adr.assemble_helmholtz(g, P.omega, P.kappa, P.gamma)
    js = g.index(P.src)
    row, ref = Ar.getrow(js).toarray().ravel(), H.getrow(js).toarray().ravel()
    assert np.abs(row - ref).max() <= 1e-12 * np.abs(ref).max()
    # away from the source the rescaled central matrix differs from H by O((w h)^2) per entry, not O(1)
    far = [j for j in range(g.N) if np.abs(np.array(g.coords(j)) - np.array(P.src)).max() > 3][:50]
    for j in far:
        d = np.abs(Ar.getrow(j).toarray().ravel() - H.getrow(j).toarray().ravel()).max()
        assert d <= 0.5 * np.abs(H.getrow(j).toarray()).max()


def test_stage2_preconditioner_is_shifted_laplacian_at_tau_zero():
    P, g = _marine()
    z = np.zeros(g.N)
    Hs = twostage.shifted_rescaled_central(g, P.src, P.omega, P.kappa, P.gamma, z, 0.2)
    H = adr.assemble_helmholtz(g, P.omega, P.kappa, P.gamma)
    ref = H - 1j * 0.2 * P.omega ** 2 * sp.diags(P.kappa ** 2)
    assert abs(Hs - ref).max() <= 1e-12 * abs(H).max()


@pytest.mark.parametrize("make", [lambda: _marine(), lambda: _marine((37, 21))])
def test_two_stage_solves_central_system(make):
    P, g = make()
    u, a, (its1, res1), (its2, res2) = twostage.two_stage_central(
        g, P.src, P.omega, P.kappa, P.gamma, P.tau1, PRM, levels=3, alpha=0.2, tol=1e-11, maxit=400)
    q_hat = adr.point_source_rhs(g, P.src)
    Ac = adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, "cen")
    a_direct = spla.spsolve(Ac.tocsc(), q_hat)
    assert np.linalg.norm(a - a_direct) <= 1e-8 * np.linalg.norm(a_direct)
    res_a = np.linalg.norm(q_hat - Ac @ a) / np.linalg.norm(q_hat)
    assert res2 <= 1e-11 and abs(res_a - res2) <= 1e-13
    m = twostage.phase(g, P.src, P.omega, P.tau1)
    assert np.allclose(u, m * a, rtol=1e-14, atol=0)
    # stage 1's stop rule on Eq. 1up
    assert its1 <= 5 and (its1 == 5 or res1 <= 1e-2)


def test_stage1_warm_start_reduces_stage2_work():
    """The global approximation of stage 1 is a better start than zero for
    the shifted-Laplacian stage (Sec. 3.2)."""
    P, g = _marine((65, 65))
    _, _, _, (its2, _) = twostage.two_stage_central(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, PRM, levels=3,
                                                     tol=1e-8, maxit=400)
    m = twostage.phase(g, P.src, P.omega, P.tau1)
    A2 = twostage.rescaled(adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, "cen"), m)
    hier = mg.build_hierarchy(twostage.shifted_rescaled_central(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, 0.2),
                              P.n, 3)
    q = m * adr.point_source_rhs(g, P.src)
    _, its_cold, _, _ = krylov.fgmres(A2, q, lambda v: mg.cycle(hier, v, PRM), tol=1e-8, restart=5, maxit=400)
    assert its2 < its_cold
