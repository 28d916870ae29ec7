"""ADR amplitude discretisation, restated row by row in FP64 (oracle).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Problem (paper convention, Sec. 1 and Eq. new_u):  u = a exp(-i w tau) with
    Delta a - 2 i w grad(tau).grad(a) - i w (Delta tau) a
            - w^2 (|grad tau|^2 - kappa^2) a - i w gamma kappa^2 a = q_hat,
    q_hat = q exp(+i w tau).                                   (Eq. ADR)
The absorbing term -i w gamma kappa^2 is the attenuation of the Helmholtz
equation of Sec. 1, kept as a mass term (Sec. 2.2.1).

Readings taken where the paper is silent or garbled (each is listed in the
design notes):
  R1  Eq. BCADR lacks the factor a; read n.grad(a) - i w (n.grad tau) a = 0.
      It is imposed on every face with a ghost node eliminated by the
      central difference:  a_{b+s} = a_{b-s} + s 2 h i w (d tau)_b a_b
      (s = +-1 the outward direction along the axis).
  R2  The averaging mass of Sec. 2.3 is applied per axis:
      -i w sum_d (d_dd tau)_j (a_{j+e_d} + a_{j-e_d}) / 2.
  R3  Delta tau is split per axis with Eq. travel_time_coeff:
      d_dd tau = tau1 d_dd tau0 + 2 d_d tau0 d_d tau1 + tau0 d_dd tau1.
  R4  At the source node tau0 has no derivative; that row is the row of
      M^{-1} H M (Eq. helmADR2, d dimensions, tau(x0) = 0), H with its own
      Neumann ghost u_{-1} = u_{+1}.
  R5  "Immediate neighbourhood of the source" (Sec. 2.2) = Chebyshev
      distance <= near_radius (default 1, the literal "distance of one node");
      those rows use central advection.  With radius 1 the second-order
      upwind rows two nodes away still reach the singular source node; radius
      2 keeps every upwind stencil off it (see the accuracy tests).
  R6  Where an upwind stencil would need a node off the grid, the row uses
      central advection along that axis instead (with the ghost of R1 on the
      boundary itself).  d_d tau == 0 exactly also takes the central form
      (its coefficient is then zero).
  R7  First-order upwind (Eq. 1up, not written out in the paper):
      tau' > 0: tau'(a_j - a_{j-1})/h;  tau' < 0: tau'(a_{j+1} - a_j)/h.
  R8  Central ADR (H_cen) switches to second-order upwind on boundary nodes
      (Sec. 2.2.1), then falls back as in R6.
  R9  The point source is q = delta_{x0} / prod(h_d) (Sec. 4.1 gives 1/h^2 in
      2D), so q_hat(x0) = 1 / prod(h_d) because tau(x0) = 0.
"""
from __future__ import annotations

import math
from collections import defaultdict

import numpy as np
import scipy.sparse as sp


class Grid:
    """Nodal regular grid; node (i0, i1[, i2]) lives at i0 + n0*(i1 + n1*i2)."""

    def __init__(self, n, h):
        self.n = tuple(int(v) for v in n)
        self.h = tuple(float(v) for v in h)
        self.dim = len(self.n)
        self.N = int(np.prod(self.n))
        self.stride = [1]
        for d in range(1, self.dim):
            self.stride.append(self.stride[-1] * self.n[d - 1])

    def index(self, i):
        return sum(int(i[d]) * self.stride[d] for d in range(self.dim))

    def coords(self, j):
        out = []
        for d in range(self.dim):
            out.append(j % self.n[d])
            j //= self.n[d]
        return tuple(out)

    def inside(self, i):
        return all(0 <= i[d] < self.n[d] for d in range(self.dim))

    def shifted(self, i, d, k):
        """Multi-index i moved by k nodes along axis d."""
        out = list(i)
        out[d] += k
        return tuple(out)


# ---------------------------------------------------------------------------
# Travel-time coefficients (Eq. travel_time_coeff)
# ---------------------------------------------------------------------------

class PlainTau:
    """A travel time given as plain nodal values tau instead of the factor
    tau1 of tau = tau0 tau1.  Wherever a function below takes `tau1`, a
    PlainTau may be passed: the coefficients then take d_d tau and d_dd tau by
    the same finite differences of tau itself (central inside, one-sided on
    the boundary) that the factored form applies to tau1, instead of
    Eq. travel_time_coeff's product rule with the analytic tau0.  Next to the
    source, where tau has its conical kink, these differences are only first
    order accurate; the factored form avoids that (Sec. 2.1)."""

    def __init__(self, values):
        self.values = np.asarray(values, dtype=np.float64)


def tau0_derivatives(grid, src, i):
    """tau0 = |x - x0| and its analytic first and second derivatives per axis."""
    dx = [(i[d] - src[d]) * grid.h[d] for d in range(grid.dim)]
    r = math.sqrt(sum(v * v for v in dx))
    if r == 0.0:
        return 0.0, [0.0] * grid.dim, [0.0] * grid.dim
    first = [dx[d] / r for d in range(grid.dim)]
    second = [(1.0 - (dx[d] / r) ** 2) / r for d in range(grid.dim)]
    return r, first, second


def tau1_first_derivative(grid, tau1, i, d):
    """d tau1 / d x_d: central difference inside, first-order one-sided on the boundary."""
    h = grid.h[d]
    k = i[d]
    n = grid.n[d]
    at = lambda m: tau1[grid.index(grid.shifted(i, d, m - k))]
    if k == 0:
        return (at(1) - at(0)) / h
    if k == n - 1:
        return (at(n - 1) - at(n - 2)) / h
    return (at(k + 1) - at(k - 1)) / (2.0 * h)


def tau1_second_derivative(grid, tau1, i, d):
    """d^2 tau1 / d x_d^2: central inside, second-order one-sided on the boundary.

    One-sided rule at the low end: (2 f0 - 5 f1 + 4 f2 - f3) / h^2 (mirrored
    at the high end); it is exact for cubics.
    """
    h = grid.h[d]
    k = i[d]
    n = grid.n[d]
    at = lambda m: tau1[grid.index(grid.shifted(i, d, m - k))]
    if k == 0:
        return (2.0 * at(0) - 5.0 * at(1) + 4.0 * at(2) - at(3)) / (h * h)
    if k == n - 1:
        return (2.0 * at(n - 1) - 5.0 * at(n - 2) + 4.0 * at(n - 3) - at(n - 4)) / (h * h)
    return (at(k + 1) - 2.0 * at(k) + at(k - 1)) / (h * h)


def node_coefficients(grid, src, omega, kappa, gamma, tau1, j):
    """Coefficients of Eq. ADR at node j.

    Returns (tau, g, t, rho): tau = tau0 tau1, g_d = d_d tau, t_d = d_dd tau
    (reading R3) and the reaction rho = w^2 (kappa^2 - |grad tau|^2)
    - i w gamma kappa^2.
    """
    i = grid.coords(j)
    if isinstance(tau1, PlainTau):                  # d tau and d^2 tau by differences of tau itself
        tv = tau1.values
        g = [tau1_first_derivative(grid, tv, i, d) for d in range(grid.dim)]
        t = [tau1_second_derivative(grid, tv, i, d) for d in range(grid.dim)]
        k2 = kappa[j] * kappa[j]
        grad2 = sum(v * v for v in g)
        return tv[j], g, t, omega * omega * (k2 - grad2) - 1j * omega * gamma[j] * k2
    r, d0, dd0 = tau0_derivatives(grid, src, i)
    t1 = tau1[j]
    g = []
    t = []
    for d in range(grid.dim):
        d1 = tau1_first_derivative(grid, tau1, i, d)
        dd1 = tau1_second_derivative(grid, tau1, i, d)
        g.append(r * d1 + t1 * d0[d])
        t.append(t1 * dd0[d] + 2.0 * d0[d] * d1 + r * dd1)
    k2 = kappa[j] * kappa[j]
    grad2 = sum(v * v for v in g)
    rho = omega * omega * (k2 - grad2) - 1j * omega * gamma[j] * k2
    return r * t1, g, t, rho


def travel_time(grid, src, tau1):
    """tau = tau0 * tau1 at every node (a PlainTau: its values)."""
    if isinstance(tau1, PlainTau):
        return tau1.values.copy()
    out = np.empty(grid.N)
    for j in range(grid.N):
        r, _, _ = tau0_derivatives(grid, src, grid.coords(j))
        out[j] = r * tau1[j]
    return out


# ---------------------------------------------------------------------------
# Rows of the discrete operators
# ---------------------------------------------------------------------------

def _central(h):
    return {+1: 1.0 / (2.0 * h), -1: -1.0 / (2.0 * h)}


def _upwind2(g, h):
    """Second-order upwind difference of Eq. londUpwindDiff."""
    if g > 0:
        return {0: 3.0 / (2.0 * h), -1: -4.0 / (2.0 * h), -2: 1.0 / (2.0 * h)}
    return {0: -3.0 / (2.0 * h), +1: 4.0 / (2.0 * h), +2: -1.0 / (2.0 * h)}


def _upwind1(g, h):
    """First-order upwind difference (reading R7)."""
    if g > 0:
        return {0: 1.0 / h, -1: -1.0 / h}
    return {0: -1.0 / h, +1: 1.0 / h}


def advection_stencil(scheme, g, h, k, n, near_source):
    """Weights of the difference D_d a along one axis, keyed by node offset."""
    if near_source or g == 0.0:
        return _central(h)
    if scheme == "2up":
        st = _upwind2(g, h)
    elif scheme == "1up":
        st = _upwind1(g, h)
    elif scheme == "cen":
        if 0 < k < n - 1:
            return _central(h)
        st = _upwind2(g, h)          # reading R8
    else:
        raise ValueError(scheme)
    if all(0 <= k + off < n for off in st):
        return st
    return _central(h)               # reading R6


def source_row(grid, src, omega, kappa, gamma, tau1):
    """Row of M^{-1} H M at the source node (reading R4, Eq. helmADR2)."""
    j = grid.index(src)
    row = defaultdict(complex)

    def tau_at(i):
        if isinstance(tau1, PlainTau):
            return tau1.values[grid.index(i)]
        r, _, _ = tau0_derivatives(grid, src, i)
        return r * tau1[grid.index(i)]

    tau_s = tau_at(src)          # 0 for the factored form (tau0 vanishes at the source)
    for d in range(grid.dim):
        h2 = grid.h[d] ** 2
        for s in (+1, -1):
            nb = grid.shifted(src, d, s)
            if not grid.inside(nb):
                nb = grid.shifted(src, d, -s)      # Neumann ghost of H: u_{b+s} = u_{b-s}
            row[grid.index(nb)] += np.exp(1j * omega * (tau_s - tau_at(nb))) / h2
            row[j] += -1.0 / h2
    k2 = kappa[j] ** 2
    row[j] += omega * omega * k2 - 1j * omega * gamma[j] * k2
    return dict(row)


def helmholtz_row(grid, omega, kappa, gamma, j):
    """Row of the standard 5/7-point Helmholtz matrix H with Neumann ghosts."""
    i = grid.coords(j)
    row = defaultdict(complex)
    for d in range(grid.dim):
        h2 = grid.h[d] ** 2
        for s in (+1, -1):
            nb = grid.shifted(i, d, s)
            if not grid.inside(nb):
                nb = grid.shifted(i, d, -s)
            row[grid.index(nb)] += 1.0 / h2
            row[j] += -1.0 / h2
    k2 = kappa[j] ** 2
    row[j] += omega * omega * k2 - 1j * omega * gamma[j] * k2
    return dict(row)


def adr_row(grid, src, omega, kappa, gamma, tau1, j, scheme, near_radius=1):
    """Row j of H_hat for scheme '2up', '1up' or 'cen' as {column: value}."""
    i = grid.coords(j)
    if tuple(i) == tuple(src):
        return source_row(grid, src, omega, kappa, gamma, tau1)
    _, g, t, rho = node_coefficients(grid, src, omega, kappa, gamma, tau1, j)
    near = max(abs(i[d] - src[d]) for d in range(grid.dim)) <= near_radius      # reading R5
    row = defaultdict(complex)
    for d in range(grid.dim):
        h = grid.h[d]

        def add(offset, value):
            """Add value * a_{i + offset e_d}; an off-grid node becomes its ghost (R1)."""
            nb = grid.shifted(i, d, offset)
            if grid.inside(nb):
                row[grid.index(nb)] += value
                return
            s = offset                          # only offsets +-1 can leave the grid
            assert abs(s) == 1
            row[grid.index(grid.shifted(i, d, -s))] += value
            row[j] += value * s * 2.0 * h * 1j * omega * g[d]

        # Laplacian
        add(+1, 1.0 / (h * h))
        add(-1, 1.0 / (h * h))
        row[j] += -2.0 / (h * h)
        # -i w (d_dd tau) * average of the two neighbours  (R2)
        add(+1, -0.5j * omega * t[d])
        add(-1, -0.5j * omega * t[d])
        # -2 i w (d_d tau) D_d a
        for off, w in advection_stencil(scheme, g[d], h, i[d], grid.n[d], near).items():
            if off == 0:
                row[j] += -2j * omega * g[d] * w
            else:
                add(off, -2j * omega * g[d] * w)
    row[j] += rho
    return dict(row)


def _assemble(grid, rows):
    r, c, v = [], [], []
    for j in range(grid.N):
        for col, val in rows(j).items():
            r.append(j)
            c.append(col)
            v.append(val)
    return sp.csr_matrix((np.array(v, dtype=np.complex128), (r, c)), shape=(grid.N, grid.N))


def assemble_adr(grid, src, omega, kappa, gamma, tau1, scheme, near_radius=1):
    """Sparse H_hat (Eqs. ADRLinSystemCentral / ADRLinSystemUpwind / 1up)."""
    return _assemble(grid, lambda j: adr_row(grid, src, omega, kappa, gamma, tau1, j, scheme, near_radius))


def assemble_helmholtz(grid, omega, kappa, gamma):
    """Sparse standard Helmholtz matrix H (Eq. HelmholtzLinSystem)."""
    return _assemble(grid, lambda j: helmholtz_row(grid, omega, kappa, gamma, j))


def assemble_preconditioner(grid, src, omega, kappa, gamma, tau1, beta=0.25, near_radius=1, shift=0.0):
    """(1 - beta) H_2up + beta H_1up  (Eq. precADRup), minus i shift w^2 kappa^2
    on the diagonal: the complex shift of Eq. shift (with tau = 0 and
    shift = alpha this is the shifted-Laplacian preconditioner)."""
    a2 = assemble_adr(grid, src, omega, kappa, gamma, tau1, "2up", near_radius)
    a1 = assemble_adr(grid, src, omega, kappa, gamma, tau1, "1up", near_radius)
    A = (1.0 - beta) * a2 + beta * a1
    if shift:
        A = A - 1j * shift * omega * omega * sp.diags(np.asarray(kappa, dtype=float) ** 2)
    return A.tocsr()


def point_source_rhs(grid, src):
    """q_hat = delta_{x0} / prod(h) (reading R9)."""
    q = np.zeros(grid.N, dtype=np.complex128)
    q[grid.index(src)] = 1.0 / float(np.prod(grid.h))
    return q


def reconstruct(grid, src, omega, tau1, a):
    """u = a exp(-i w tau), tau = tau0 tau1 (Eq. new_u)."""
    tau = travel_time(grid, src, tau1)
    return np.asarray(a) * np.exp(-1j * omega * tau)


def phase_matrix(grid, src, omega, tau1):
    """Diagonal M with M_jj = exp(-i w tau_j) (Eq. matrix_rescaling)."""
    return sp.diags(np.exp(-1j * omega * travel_time(grid, src, tau1)))
