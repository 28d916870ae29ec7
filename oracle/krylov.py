"""Flexible GMRES (oracle).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

The paper wraps its multigrid cycle in flexible GMRES (Sec. 3.1, Sec. 4.2),
right-preconditioned, from a zero initial guess, stopping on the relative
residual.  Readings (also in the design notes):
  K1  Orthogonalisation is classical Gram-Schmidt applied twice (the paper is
      silent); the least-squares problem is reduced with Givens rotations.
  K2  Inside a cycle the stop test uses the Givens residual estimate
      |g_{j+1}| / |b|; at the end of every cycle the residual b - A x is
      recomputed explicitly and the solve stops when it meets the tolerance
      or the iteration budget is spent.
  K3  A cycle ends after `restart` iterations, on convergence of the
      estimate, on an exact breakdown, or when the budget is spent.
  K4  With reorth_eta < 1 the second Gram-Schmidt pass of K1 runs only when
      the first pass cancelled |w| below reorth_eta |w| (the test of Daniel,
      Gragg, Kaufman and Stewart, 1976, compared on squared norms); a single
      classical pass otherwise.  reorth_eta >= 1 (or None) is K1 unchanged.
"""
from __future__ import annotations

import numpy as np

from .multigrid import back_substitution, cgs2, givens


def cgs_selective(V, w, eta):
    """Classical Gram-Schmidt against the columns of V, repeated only when the
    first pass leaves less than eta |w| (reading K4).  Returns (h, w)."""
    s2 = np.vdot(w, w).real
    h = V.conj().T @ w
    w = w - V @ h
    if np.vdot(w, w).real >= eta * eta * s2:
        return h, w
    h2 = V.conj().T @ w
    w = w - V @ h2
    return h + h2, w


def fgmres(A, b, precond, x0=None, tol=1e-8, restart=20, maxit=500, reorth_eta=None):
    """Solve A x = b.  Returns (x, iterations, final relative residual, history).

    `history` holds the estimate |g_{j+1}|/|b| after every iteration.
    reorth_eta: None or >= 1 for CGS2 (K1), else the selective test of K4.
    """
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n, dtype=np.complex128), 0, 0.0, []
    history = []
    its = 0
    r = b - A @ x
    beta = np.linalg.norm(r)
    while beta > tol * bnorm and its < maxit:
        V = np.zeros((n, restart + 1), dtype=np.complex128)
        Z = np.zeros((n, restart), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        V[:, 0] = r / beta
        g[0] = beta
        k = 0
        for j in range(restart):
            Z[:, j] = precond(V[:, j])
            w = A @ Z[:, j]
            if reorth_eta is None or reorth_eta >= 1.0:
                hcol, w = cgs2(V[:, : j + 1], w)
            else:
                hcol, w = cgs_selective(V[:, : j + 1], w, reorth_eta)
            H[: j + 1, j] = hcol
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):
                a, bb = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * bb
                H[i + 1, j] = -np.conj(sn[i]) * a + cs[i] * bb
            hn = H[j + 1, j].real
            cs[j], sn[j], H[j, j] = givens(H[j, j], H[j + 1, j])
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            if hn == 0.0:
                break
            V[:, j + 1] = w / hn
            if abs(g[j + 1]) <= tol * bnorm or its >= maxit:
                break
        y = back_substitution(H[:k, :k], g[:k])
        x = x + Z[:, :k] @ y
        r = b - A @ x
        beta = np.linalg.norm(r)
    return x, its, beta / bnorm, history
