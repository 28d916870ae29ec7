"""Receiver misfit and its slowness gradient by the adjoint state (oracle).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

The paper stops at the forward solve; the gradient here is the textbook
adjoint-state derivative of J(kappa) = sum_s 1/2 |R u_s - d_s|^2 through the
discrete system of the oracle's own assembly, with the travel time and the
absorbing profile held fixed:
    H a = q_hat,   u = M a,   M = diag(exp(-i w tau))            (Eq. new_u)
    dJ/dkappa_j = Re( (R u - d)^H R M da/dkappa_j )
                = -Re( lambda^H (dH/dkappa_j) a ),   H^H lambda = M^H R^T (R u - d).
kappa appears in H only in the reaction diagonal w^2 kappa^2 - i w gamma
kappa^2 (Eq. ADR, also in the source row of reading R4), so dH/dkappa_j is the
single diagonal entry 2 w^2 kappa_j - 2 i w gamma_j kappa_j.  The adjoint is
the conjugate transpose of the assembled CSR matrix; both solves are direct.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import adr


def forward_wavefield(grid, src, omega, kappa, gamma, tau1, near_radius=1):
    """(H, a, u) for one point source: direct solve of H_2up a = q_hat, u = M a."""
    H = adr.assemble_adr(grid, src, omega, kappa, gamma, tau1, "2up", near_radius).tocsc()
    a = spla.spsolve(H, adr.point_source_rhs(grid, src))
    return H, a, adr.reconstruct(grid, src, omega, tau1, a)


def misfit(grid, sources, omega, kappa, gamma, tau1s, receivers, data, near_radius=1):
    """J = sum_s 1/2 |u_s[receivers] - d_s|^2."""
    J = 0.0
    for src, tau1, d in zip(sources, tau1s, data):
        _, _, u = forward_wavefield(grid, src, omega, kappa, gamma, tau1, near_radius)
        r = u[receivers] - d
        J += 0.5 * float(np.vdot(r, r).real)
    return J


def misfit_gradient(grid, sources, omega, kappa, gamma, tau1s, receivers, data, near_radius=1):
    """(J, dJ/dkappa) by one forward and one adjoint direct solve per source."""
    receivers = np.asarray(receivers, dtype=np.int64)
    J = 0.0
    g = np.zeros(grid.N)
    dHdk = 2.0 * omega * omega * kappa - 2j * omega * gamma * kappa
    for src, tau1, d in zip(sources, tau1s, data):
        H, a, u = forward_wavefield(grid, src, omega, kappa, gamma, tau1, near_radius)
        r = u[receivers] - d
        J += 0.5 * float(np.vdot(r, r).real)
        tau = adr.travel_time(grid, src, tau1)
        f = np.zeros(grid.N, dtype=np.complex128)
        np.add.at(f, receivers, np.exp(1j * omega * tau[receivers]) * r)
        lam = spla.spsolve(H.conj().T.tocsc(), f)
        g -= (np.conj(lam) * dHdk * a).real
    return J, g
