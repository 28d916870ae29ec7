"""Geometric multigrid with Galerkin coarse operators (oracle).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

* P is bilinear (2D) / trilinear (3D) interpolation on nodal grids (Sec. 3.1);
  the restriction is its plain transpose P^T, unscaled (Sec. 3, Alg. TwoGrid).
* Coarse operators are Galerkin products A_c = P^T A P (Eq. coarseGridMatrix).
* Relaxation is damped Jacobi x <- x + w D^{-1} (b - A x) with a weight per
  level, or one step of Jacobi-preconditioned GMRES, which is Jacobi with the
  complex weight minimising the residual (Sec. 3.1; the paper relaxes with
  Jacobi-preconditioned GMRES, l+1 sweeps on level l, Sec. 4.2).
* The cycle is the two-grid cycle of Alg. TwoGrid applied recursively once
  (a V-cycle) or with an inner flexible GMRES on the coarse levels
  (Alg. Kcycle); the coarsest level is solved inexactly by a fixed number of
  Jacobi-preconditioned GMRES iterations started from zero (Sec. 3.1, Sec. 4.2:
  ten iterations instead of a factorisation).

Readings (also in the design notes):
  M1  A level can be coarsened when every axis has an odd node count >= 5;
      the coarse grid keeps every other node.
  M2  The coarsest GMRES is right-preconditioned by D = diag(A), uses
      classical Gram-Schmidt applied twice and stops early only on an exact
      breakdown (h_{j+1,j} == 0).  With coarse_reorth_eta < 1 the second
      pass runs only when the first one left less than that fraction of |w|
      (the selective test of the outer iteration, reading K4 of krylov).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def interpolation_1d(nf):
    """Linear interpolation from (nf-1)/2+1 coarse nodes to nf fine nodes."""
    nc = (nf - 1) // 2 + 1
    rows, cols, vals = [], [], []
    for i in range(nf):
        if i % 2 == 0:
            rows.append(i); cols.append(i // 2); vals.append(1.0)
        else:
            rows += [i, i]; cols += [i // 2, i // 2 + 1]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def prolongation(n_fine):
    """Tensor-product interpolation; axis 0 is the fastest index."""
    P = None
    for nf in n_fine:                      # kron(P_last, ..., P_0)
        p1 = interpolation_1d(nf)
        P = p1 if P is None else sp.kron(p1, P, format="csr")
    return P.tocsr()


def can_coarsen(n):
    """Reading M1."""
    return all(v % 2 == 1 and v >= 5 for v in n)


def coarse_shape(n):
    return tuple((v - 1) // 2 + 1 for v in n)


def build_hierarchy(A1, n, levels):
    """[{A, n, P (to the next coarser level), dinv}] with A_{l+1} = P^T A_l P."""
    out = [{"A": A1.tocsr(), "n": tuple(n)}]
    while len(out) < levels and can_coarsen(out[-1]["n"]):
        lv = out[-1]
        P = prolongation(lv["n"])
        lv["P"] = P
        Ac = (P.T @ lv["A"] @ P).tocsr()
        out.append({"A": Ac, "n": coarse_shape(lv["n"])})
    for lv in out:
        lv["dinv"] = 1.0 / lv["A"].diagonal()
    return out


def jacobi(A, dinv, x, b, weight):
    """One damped-Jacobi sweep."""
    return x + weight * dinv * (b - A @ x)


def givens(a, b):
    """Complex Givens rotation (c real) with [c s; -conj(s) c] [a; b] = [r; 0]."""
    if b == 0:
        return 1.0, 0.0 + 0.0j, a
    if a == 0:
        return 0.0, 1.0 + 0.0j, b
    nu = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    c = abs(a) / nu
    s = (a / abs(a)) * np.conj(b) / nu
    return c, s, (a / abs(a)) * nu


def cgs2(V, w):
    """Classical Gram-Schmidt against the columns of V, applied twice."""
    h = V.conj().T @ w
    w = w - V @ h
    h2 = V.conj().T @ w
    w = w - V @ h2
    return h + h2, w


def coarse_gmres(A, dinv, b, iterations, reorth_eta=None):
    """Fixed-count GMRES from x = 0, right-preconditioned by Jacobi (reading M2);
    reorth_eta < 1: the selective second Gram-Schmidt pass."""
    from .krylov import cgs_selective
    n = b.shape[0]
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros(n, dtype=np.complex128)
    V = np.zeros((n, iterations + 1), dtype=np.complex128)
    H = np.zeros((iterations + 1, iterations), dtype=np.complex128)
    cs = np.zeros(iterations)
    sn = np.zeros(iterations, dtype=np.complex128)
    g = np.zeros(iterations + 1, dtype=np.complex128)
    V[:, 0] = b / beta
    g[0] = beta
    k = 0
    for j in range(iterations):
        w = A @ (dinv * V[:, j])
        if reorth_eta is None or reorth_eta >= 1.0:
            hcol, w = cgs2(V[:, : j + 1], w)
        else:
            hcol, w = cgs_selective(V[:, : j + 1], w, reorth_eta)
        H[: j + 1, j] = hcol
        H[j + 1, j] = np.linalg.norm(w)
        for i in range(j):                         # earlier rotations
            a, bb = H[i, j], H[i + 1, j]
            H[i, j] = cs[i] * a + sn[i] * bb
            H[i + 1, j] = -np.conj(sn[i]) * a + cs[i] * bb
        hn = H[j + 1, j].real
        cs[j], sn[j], H[j, j] = givens(H[j, j], H[j + 1, j])
        H[j + 1, j] = 0.0
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        if hn == 0.0:
            break
        V[:, j + 1] = w / hn
    y = back_substitution(H[:k, :k], g[:k])
    return dinv * (V[:, :k] @ y)


def back_substitution(R, g):
    """Solve the upper-triangular system R y = g."""
    k = R.shape[0]
    y = np.zeros(k, dtype=np.complex128)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - R[i, i + 1:] @ y[i + 1:]) / R[i, i]
    return y


def vcycle(hier, b, weights, nu1=1, nu2=1, coarse_iterations=10, level=0):
    """One V(nu1, nu2) cycle from a zero initial guess (Alg. TwoGrid, recursive)."""
    lv = hier[level]
    A, dinv = lv["A"], lv["dinv"]
    if level == len(hier) - 1:
        return coarse_gmres(A, dinv, b, coarse_iterations)
    x = np.zeros_like(b)
    for _ in range(nu1):
        x = jacobi(A, dinv, x, b, weights[level])
    r = b - A @ x
    bc = lv["P"].T @ r
    ec = vcycle(hier, bc, weights, nu1, nu2, coarse_iterations, level + 1)
    x = x + lv["P"] @ ec
    for _ in range(nu2):
        x = jacobi(A, dinv, x, b, weights[level])
    return x


# ---------------------------------------------------------------------------
# Cycle variants (Sec. 3.1, Alg. TwoGrid, Alg. Kcycle)
# ---------------------------------------------------------------------------
class CycleParams:
    """Plain settings of the multigrid cycle.

    cycle: 'V' (Alg. TwoGrid recursively) or 'K' (Alg. Kcycle);
    relax: 'jacobi' (fixed weight per level) or 'mr' (one step of
    Jacobi-preconditioned GMRES, i.e. Jacobi with the complex weight that
    minimises the residual, Sec. 3.1); pre/post: sweeps per level;
    coarse_iterations: fixed GMRES steps on the coarsest grid;
    kcycle_iterations: inner FGMRES steps of the K-cycle;
    kcycle_threshold: the inner FGMRES stops early once its residual is at
    most this fraction of the restricted residual it started from (Sec. 4.2
    uses 0.1 for the coarse grids: some cycles then make one recursive call
    instead of two); 0 runs the fixed count;
    coarse_reorth_eta: None (classical Gram-Schmidt twice in the coarsest
    GMRES) or the selective second pass's threshold (reading M2).
    """

    def __init__(self, cycle="K", relax="mr", pre=None, post=None, weights=None,
                 coarse_iterations=10, kcycle_iterations=2, kcycle_threshold=0.0, coarse_reorth_eta=None):
        self.cycle = cycle
        self.relax = relax
        self.pre = list(pre) if pre is not None else [l + 2 for l in range(8)]
        self.post = list(post) if post is not None else [l + 2 for l in range(8)]
        self.weights = list(weights) if weights is not None else [0.5] * 8
        self.coarse_iterations = coarse_iterations
        self.kcycle_iterations = kcycle_iterations
        self.kcycle_threshold = kcycle_threshold
        self.coarse_reorth_eta = coarse_reorth_eta


def relax_mr(A, dinv, x, b):
    """One GMRES step on A e = r from e = 0, right-preconditioned by Jacobi.

    The one-dimensional least-squares problem min |r - alpha A D^{-1} r| has
    the closed-form solution alpha = (w^H r) / (w^H w) with w = A D^{-1} r.
    """
    r = b - A @ x
    z = dinv * r
    w = A @ z
    den = np.vdot(w, w).real
    alpha = np.vdot(w, r) / den if den > 0 else 0.0
    return x + alpha * z


def _relax(lv, x, b, params, level):
    if params.relax == "jacobi":
        return jacobi(lv["A"], lv["dinv"], x, b, params.weights[level])
    return relax_mr(lv["A"], lv["dinv"], x, b)


def fixed_fgmres(A, b, precond, iterations):
    """`iterations` steps of flexible GMRES from zero, no restart and no early stop."""
    from .krylov import fgmres
    x, _, _, _ = fgmres(A, b, precond, tol=0.0, restart=iterations, maxit=iterations)
    return x


def kcycle_fgmres(A, b, precond, iterations, threshold):
    """The inner solve of Alg. Kcycle: flexible GMRES from zero (one Arnoldi
    cycle, classical Gram-Schmidt applied twice, Givens rotations) that stops
    after step j when the least-squares residual |g_{j+1}| is at most
    threshold * |b|, and after `iterations` steps otherwise (Sec. 4.2: the
    threshold 0.1 lets some cycles skip their second recursive call).
    Returns (x, steps taken)."""
    n = b.shape[0]
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros(n, dtype=np.complex128), 0
    V = np.zeros((n, iterations + 1), dtype=np.complex128)
    Z = np.zeros((n, iterations), dtype=np.complex128)
    H = np.zeros((iterations + 1, iterations), dtype=np.complex128)
    cs = np.zeros(iterations)
    sn = np.zeros(iterations, dtype=np.complex128)
    g = np.zeros(iterations + 1, dtype=np.complex128)
    V[:, 0] = b / beta
    g[0] = beta
    k = 0
    for j in range(iterations):
        Z[:, j] = precond(V[:, j])
        hcol, w = cgs2(V[:, : j + 1], A @ Z[:, j])
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
        k = j + 1
        if hn == 0.0 or abs(g[j + 1]) <= threshold * beta:
            break
        V[:, j + 1] = w / hn
    y = back_substitution(H[:k, :k], g[:k])
    return Z[:, :k] @ y, k


def cycle(hier, b, params, level=0):
    """x = B_l^{-1} b from a zero guess with the cycle selected by `params`."""
    lv = hier[level]
    A, dinv = lv["A"], lv["dinv"]
    if level == len(hier) - 1:
        return coarse_gmres(A, dinv, b, params.coarse_iterations, params.coarse_reorth_eta)
    x = np.zeros_like(b)
    for _ in range(params.pre[level]):
        x = _relax(lv, x, b, params, level)
    bc = lv["P"].T @ (b - A @ x)
    nxt = level + 1
    if params.cycle == "K" and nxt < len(hier) - 1 and params.kcycle_threshold > 0.0:
        xc, _ = kcycle_fgmres(hier[nxt]["A"], bc, lambda v: cycle(hier, v, params, nxt), params.kcycle_iterations,
                              params.kcycle_threshold)
    elif params.cycle == "K" and nxt < len(hier) - 1:
        xc = fixed_fgmres(hier[nxt]["A"], bc, lambda v: cycle(hier, v, params, nxt), params.kcycle_iterations)
    else:
        xc = cycle(hier, bc, params, nxt)
    x = x + lv["P"] @ xc
    for _ in range(params.post[level]):
        x = _relax(lv, x, b, params, level)
    return x
