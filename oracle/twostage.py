"""Two-stage solve of the central ADR system (Alg. ADRlong) -- oracle.

TEST INFRASTRUCTURE ONLY -- see the package docstring.

The steps, in the paper's order and notation (Sec. 3.2):
  Stage 1: a_1up = a low-accuracy solution of H_1up a = q_hat (Eq. 1up) by
           FGMRES with the multigrid cycle built on H_1up itself;
           M = diag(exp(-i w tau)), u_1up = M a_1up.
  Stage 2: H_s^cen = M H_cen M^{-1} - i w^2 alpha diag(kappa^2) (Eq. shift
           applied to the rescaled central matrix); FGMRES on
           M H_cen M^{-1} u = q (Eq. ADRcenRescaled) with the multigrid cycle
           on H_s^cen as the preconditioner, starting from u_1up.
Readings (also in the design notes):
  TS1 The stage-1 preconditioner is the cycle on H_1up (the blend of
      Eq. precADRup with beta = 1): the paper solves Eq. 1up "by Algorithm
      KrylovCycle" and notes that H_1up is handled very well by multigrid.
  TS2 Stage 1 stops after at most 5 outer FGMRES iterations or at relative
      residual 1e-2 of Eq. 1up, whichever comes first (Sec. 4.2).
  TS3 q = M q_hat, the right-hand side of H u = q for u = M a (Eq.
      matrix_rescaling read for the system); at a point source tau(x0) = 0,
      so q = q_hat.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import adr, krylov
from . import multigrid as mg


def phase(grid, src, omega, tau1):
    """Diagonal of M: exp(-i w tau) with tau = tau0 tau1 (Eq. matrix_rescaling)."""
    return np.exp(-1j * omega * adr.travel_time(grid, src, tau1))


def rescaled(Ahat, m):
    """M Ahat M^{-1} for M = diag(m)."""
    return (sp.diags(m) @ Ahat @ sp.diags(1.0 / m)).tocsr()


def shifted_rescaled_central(grid, src, omega, kappa, gamma, tau1, alpha, near_radius=1):
    """H_s^cen = M H_cen M^{-1} - i w^2 alpha diag(kappa^2) (Alg. ADRlong, stage 2)."""
    m = phase(grid, src, omega, tau1)
    Ac = adr.assemble_adr(grid, src, omega, kappa, gamma, tau1, "cen", near_radius)
    return (rescaled(Ac, m) - 1j * alpha * omega * omega * sp.diags(np.asarray(kappa, dtype=float) ** 2)).tocsr()


def two_stage_central(grid, src, omega, kappa, gamma, tau1, cycle_params, levels, alpha=0.2, stage1_tol=1e-2,
                      stage1_maxit=5, tol=1e-8, restart=5, maxit=500, reorth_eta=None, near_radius=1):
    """Alg. ADRlong.  Returns (u, a, stage-1 (iterations, residual), stage-2 (iterations, residual)).

    a = M^{-1} u is the amplitude of the central system H_cen a = q_hat; the
    stage-2 residual |q - M H_cen M^{-1} u| / |q| equals |q_hat - H_cen a| /
    |q_hat| because M is unitary."""
    n = grid.n
    q_hat = adr.point_source_rhs(grid, src)
    # Stage 1
    A1 = adr.assemble_adr(grid, src, omega, kappa, gamma, tau1, "1up", near_radius)
    hier1 = mg.build_hierarchy(A1, n, levels)
    a1, its1, res1, _ = krylov.fgmres(A1, q_hat, lambda v: mg.cycle(hier1, v, cycle_params), tol=stage1_tol,
                                      restart=restart, maxit=stage1_maxit, reorth_eta=reorth_eta)
    m = phase(grid, src, omega, tau1)
    u1 = m * a1
    # Stage 2
    Ac = adr.assemble_adr(grid, src, omega, kappa, gamma, tau1, "cen", near_radius)
    A2 = rescaled(Ac, m)
    Hs = shifted_rescaled_central(grid, src, omega, kappa, gamma, tau1, alpha, near_radius)
    hier2 = mg.build_hierarchy(Hs, n, levels)
    q = m * q_hat
    u, its2, res2, _ = krylov.fgmres(A2, q, lambda v: mg.cycle(hier2, v, cycle_params), x0=u1, tol=tol,
                                     restart=restart, maxit=maxit, reorth_eta=reorth_eta)
    return u, u / m, (its1, res1), (its2, res2)
