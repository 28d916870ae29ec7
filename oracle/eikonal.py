"""Factored-eikonal fast marching (oracle).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Solves |tau0 grad(tau1) + tau1 grad(tau0)|^2 = kappa^2 (Eq. factoredEikonal)
for tau1, with tau0 = |x - x0| and its gradient taken analytically, by fast
marching: nodes are accepted in increasing order of tau = tau0 tau1 from a
binary heap (Sec. 1, the factored eikonal discussion; the paper uses the
second-order fast marching of its reference [TH2016], which is not restated
in the paper, so the local update below is this oracle's own reading):

  E1  Along each axis the one-sided difference of tau1 points to the accepted
      face neighbour with the smaller tau.  An axis with no accepted
      neighbour contributes nothing (as in the Godunov upwind form of the
      plain eikonal), so a tentative value is never below the final one; in
      a constant medium the update is still exact (tau1 = kappa), because an
      axis along which tau0 varies always has an accepted, closer neighbour
      by the time the node is accepted.
  E2  order=2 uses (3 t_j - 4 t_nb + t_nb2) / 2h when the next node nb2 along
      the same direction is accepted and tau(nb2) <= tau(nb); nodes at
      Chebyshev distance 1 from the source always use first order (the paper
      notes that fast marching reverts to first order next to the source).
  E3  The quadratic in tau1_j takes its larger root.  If the discriminant is
      negative or the root would make tau_j smaller than the tau of a
      neighbour it used, the update retries with first-order differences and
      then drops the used axis with the largest neighbour tau; with a single
      axis left a negative discriminant is clamped to zero.
  E4  tau1(x0) = kappa(x0); heap ties are broken by the lower linear index.
"""
from __future__ import annotations

import heapq
import math

import numpy as np

from .adr import Grid, tau0_derivatives


def _solve_quadratic(terms, kappa_j):
    """Larger root of sum_d (A_d t + B_d)^2 = kappa^2, or None."""
    a2 = sum(A * A for A, _ in terms)
    a1 = 2.0 * sum(A * B for A, B in terms)
    a0 = sum(B * B for _, B in terms) - kappa_j * kappa_j
    disc = a1 * a1 - 4.0 * a2 * a0
    return a2, a1, disc


def factored_fast_marching(grid: Grid, kappa, src, order=2):
    """Return tau1 (flat array) for slowness kappa and a source at node src."""
    kappa = np.asarray(kappa, dtype=np.float64)
    N = grid.N
    tau1 = np.full(N, np.inf)
    accepted = np.zeros(N, dtype=bool)
    tau0 = np.empty(N)
    dtau0 = []
    for j in range(N):
        r, d0, _ = tau0_derivatives(grid, src, grid.coords(j))
        tau0[j] = r
        dtau0.append(d0)

    def tau(j):
        return tau0[j] * tau1[j]

    js = grid.index(src)
    tau1[js] = kappa[js]
    accepted[js] = True

    def local_update(j):
        i = grid.coords(j)
        near = max(abs(i[d] - src[d]) for d in range(grid.dim)) <= 1
        axes = []
        for d in range(grid.dim):
            best = None
            for s in (-1, +1):
                nb = grid.shifted(i, d, s)
                if not grid.inside(nb):
                    continue
                k = grid.index(nb)
                if accepted[k] and (best is None or tau(k) < best[2]):
                    best = (s, k, tau(k))
            if best is None:
                continue
            s, k, t_nb = best
            k2 = None
            nb2 = grid.shifted(i, d, 2 * s)
            if order == 2 and not near and grid.inside(nb2):
                kk = grid.index(nb2)
                if accepted[kk] and tau(kk) <= t_nb:
                    k2 = kk
            axes.append((t_nb, d, s, k, k2))
        axes.sort()
        h = grid.h
        for second in ((True, False) if order == 2 else (False,)):
            active = list(axes)
            while active:
                terms = []
                used = {a[1]: a for a in active}
                for d in range(grid.dim):
                    if d not in used:
                        continue
                    _, _, s, k, k2 = used[d]
                    if second and k2 is not None:
                        A = -s * 3.0 * tau0[j] / (2.0 * h[d]) + dtau0[j][d]
                        B = s * tau0[j] * (4.0 * tau1[k] - tau1[k2]) / (2.0 * h[d])
                    else:
                        A = -s * tau0[j] / h[d] + dtau0[j][d]
                        B = s * tau0[j] * tau1[k] / h[d]
                    terms.append((A, B))
                a2, a1, disc = _solve_quadratic(terms, kappa[j])
                if disc < 0.0 and len(active) == 1 and not second:
                    disc = 0.0
                if disc >= 0.0:
                    t = (-a1 + math.sqrt(disc)) / (2.0 * a2)
                    if all(tau0[j] * t >= a[0] for a in active) or (len(active) == 1 and not second):
                        return t
                active = active[:-1]
        return None

    heap = []

    def push_neighbours(j):
        i = grid.coords(j)
        for d in range(grid.dim):
            for s in (-1, +1):
                nb = grid.shifted(i, d, s)
                if not grid.inside(nb):
                    continue
                k = grid.index(nb)
                if accepted[k]:
                    continue
                t = local_update(k)
                if t is not None and t < tau1[k]:
                    tau1[k] = t
                    heapq.heappush(heap, (tau0[k] * t, k))

    push_neighbours(js)
    while heap:
        t, k = heapq.heappop(heap)
        if accepted[k] or t != tau0[k] * tau1[k]:
            continue
        accepted[k] = True
        push_neighbours(k)
    return tau1
