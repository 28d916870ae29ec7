"""Seeded synthetic inputs for the ADR amplitude solver.

This module builds the *problem data* only: nodal grids, velocity models,
the absorbing-layer profile gamma, source positions and frequencies.  It holds
none of the solver's arithmetic (no travel-time coefficients, no stencils, no
multigrid, no Krylov), so the CUDA path and the CPU checker can both draw
their inputs from it without sharing any of the method.

Conventions
-----------
* Arrays are flat float64 vectors of length N = prod(n), node (i0, i1[, i2])
  at linear index i0 + n0*(i1 + n1*i2): axis 0 is fastest.  The last axis is
  depth; depth index 0 is the surface.
* Units are km, s, km/s and rad/s.  The discrete problem depends only on
  omega*h*kappa and the geometry, so the choice of units is cosmetic.
* The absorbing layer follows the paper's description (Sec. 1, the attenuated
  Helmholtz equation): gamma grows quadratically from 0 to omega over about
  one wavelength towards each absorbing face.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One point-source amplitude problem on a nodal grid."""

    name: str
    n: tuple            # nodes per axis, axis 0 fastest
    h: tuple            # spacing per axis (km)
    src: tuple          # source node index per axis
    omega: float        # angular frequency (rad/s)
    kappa: np.ndarray   # slowness per node (s/km), flat
    gamma: np.ndarray   # absorbing-layer profile per node (1/s), flat
    tau1: np.ndarray | None = None   # travel-time factor when known in closed form
    layer_faces: tuple = ()          # (axis, side) pairs that carry a layer
    meta: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def N(self) -> int:
        return int(np.prod(self.n))


def node_coordinates(n, h):
    """Physical coordinates of every node, one flat array per axis."""
    grids = np.meshgrid(*[np.arange(v) * hv for v, hv in zip(n, h)], indexing="ij")
    # meshgrid(ij) gives shape n with axis 0 slowest in C order; transpose so
    # that axis 0 is fastest in the flat layout.
    return [np.ascontiguousarray(g.transpose()).reshape(-1) for g in grids]


def frequency_for_ppw(v_min: float, h_max: float, ppw: float = 10.0) -> float:
    """Angular frequency giving `ppw` points per wavelength at velocity v_min."""
    f = v_min / (ppw * h_max)
    return 2.0 * math.pi * f


def absorbing_layer(n, h, kappa, omega, faces, widths=None):
    """Quadratic absorbing profile gamma (0 inside, omega on the absorbing faces).

    Each face in `faces` ((axis, side), side 0 = low index) gets a layer one
    wavelength thick, the wavelength taken at the mean velocity over that face
    and rounded to whole cells; `widths` may override it with a cell count per
    face.  Contributions of faces that overlap (corners) add up.
    """
    n = tuple(n)
    dim = len(n)
    idx = np.meshgrid(*[np.arange(v) for v in n], indexing="ij")
    idx = [np.ascontiguousarray(g.transpose()).reshape(-1) for g in idx]
    kap = np.asarray(kappa, dtype=np.float64).reshape(-1)
    gamma = np.zeros(int(np.prod(n)), dtype=np.float64)
    used = {}
    for k, (axis, side) in enumerate(faces):
        on_face = idx[axis] == (0 if side == 0 else n[axis] - 1)
        if widths is not None:
            cells = int(widths[k])
        else:
            v_mean = float(np.mean(1.0 / kap[on_face]))
            wavelength = 2.0 * math.pi * v_mean / omega
            cells = max(1, int(round(wavelength / h[axis])))
        used[(axis, side)] = cells
        width = cells * h[axis]
        dist = (idx[axis] if side == 0 else (n[axis] - 1 - idx[axis])) * h[axis]
        inside = dist < width
        gamma[inside] += omega * ((width - dist[inside]) / width) ** 2
    return gamma, used


def all_faces(dim):
    return tuple((a, s) for a in range(dim) for s in (0, 1))


def faces_except_surface(dim):
    """Every face except the top (depth index 0), which keeps a plain Neumann condition."""
    return tuple(f for f in all_faces(dim) if f != (dim - 1, 0))


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

def constant_medium(n=(129, 129), extent=1.0, kappa0=1.0, ppw=10.0, src=None,
                    faces=None, layer_cells=None, name="constant"):
    """Unit-square (or cube) constant medium, source at the centre.

    tau1 is known in closed form: tau = kappa0 * |x - x0|, i.e. tau1 = kappa0.
    With n = 129x129 this is the 2D constant-slowness workload (h = 1/128,
    omega = 2*pi*12.8, 10 points per wavelength, layer on every face).
    """
    n = tuple(int(v) for v in n)
    dim = len(n)
    h = tuple(extent / (v - 1) for v in n)
    if src is None:
        src = tuple((v - 1) // 2 for v in n)
    kappa = np.full(int(np.prod(n)), kappa0, dtype=np.float64)
    omega = frequency_for_ppw(1.0 / kappa0, max(h), ppw)
    faces = all_faces(dim) if faces is None else tuple(faces)
    widths = None if layer_cells is None else [layer_cells] * len(faces)
    gamma, used = absorbing_layer(n, h, kappa, omega, faces, widths)
    tau1 = np.full(int(np.prod(n)), kappa0, dtype=np.float64)
    return Problem(name, n, h, tuple(src), omega, kappa, gamma, tau1, faces,
                   {"layer_cells": used, "ppw": ppw})


def _gaussian_anomalies(coords, extent, count, amplitude, rng):
    """Product of (1 + A_k exp(-|x - c_k|^2 / (2 sigma_k^2))) over `count` anomalies."""
    factor = np.ones_like(coords[0])
    params = []
    for _ in range(count):
        sign = 1.0 if rng.random() < 0.5 else -1.0
        sigma = rng.uniform(0.3, 0.8)
        centre = [rng.uniform(0.1 * e, 0.9 * e) for e in extent]
        r2 = sum((c - cc) ** 2 for c, cc in zip(coords, centre))
        factor *= 1.0 + sign * amplitude * np.exp(-r2 / (2.0 * sigma * sigma))
        params.append({"amplitude": sign * amplitude, "sigma": sigma, "centre": centre})
    return factor, params


def gradient_model(n, extent, v_top, v_bottom, anomalies, amplitude, seed,
                   src, ppw=10.0, faces=None, name="gradient"):
    """Velocity rising linearly with depth times seeded Gaussian anomalies.

    Stands in for the paper's smooth geophysical models (its 2D and 3D linear
    velocity models): long, shallow domains with velocity growing with depth.
    """
    n = tuple(int(v) for v in n)
    dim = len(n)
    h = tuple(e / (v - 1) for e, v in zip(extent, n))
    coords = node_coordinates(n, h)
    depth = coords[-1]
    v = v_top + (v_bottom - v_top) * depth / extent[-1]
    rng = np.random.default_rng(seed)
    factor, params = _gaussian_anomalies(coords, extent, anomalies, amplitude, rng)
    v = v * factor
    kappa = 1.0 / v
    omega = frequency_for_ppw(float(v.min()), max(h), ppw)
    faces = faces_except_surface(dim) if faces is None else tuple(faces)
    gamma, used = absorbing_layer(n, h, kappa, omega, faces)
    return Problem(name, n, h, tuple(src), omega, kappa, gamma, None, faces,
                   {"layer_cells": used, "ppw": ppw, "anomalies": params,
                    "v_min": float(v.min()), "v_max": float(v.max()), "seed": seed})


def marine_2d(n=(513, 513), seed=1):
    """2D 8 x 4 km model, v = 1.5 -> 4.5 km/s with depth, 3 Gaussians of +-20%.

    Source 50 m below the top centre, snapped to the nearest node.
    """
    extent = (8.0, 4.0)
    h_z = extent[1] / (n[1] - 1)
    src = ((n[0] - 1) // 2, int(round(0.05 / h_z)))
    return gradient_model(n, extent, 1.5, 4.5, 3, 0.20, seed, src,
                          name=f"gradient2d_{n[0]}x{n[1]}")


def layered_3d(n=(257, 257, 129), seed=2, src=None):
    """3D 6.4 x 6.4 x 3.2 km model, v = 1.5 -> 5.0 km/s with depth, 5 Gaussians of +-15%.

    With n = 257x257x129 the spacing is 25 m on every axis; the default
    source sits at the lateral centre, two nodes below the surface.
    """
    extent = (6.4, 6.4, 3.2)
    if src is None:
        src = ((n[0] - 1) // 2, (n[1] - 1) // 2, min(2, n[2] - 1))
    return gradient_model(n, extent, 1.5, 5.0, 5, 0.15, seed, src,
                          name=f"layered3d_{n[0]}x{n[1]}x{n[2]}")


def linear_velocity(n, extent, v0, grad, src, ppw=10.0, faces=None, name="linear"):
    """v = v0 + grad*depth, no anomalies (the paper's linear velocity model family)."""
    n = tuple(int(v) for v in n)
    dim = len(n)
    h = tuple(e / (v - 1) for e, v in zip(extent, n))
    coords = node_coordinates(n, h)
    v = v0 + grad * coords[-1]
    kappa = 1.0 / v
    omega = frequency_for_ppw(float(v.min()), max(h), ppw)
    faces = faces_except_surface(dim) if faces is None else tuple(faces)
    gamma, used = absorbing_layer(n, h, kappa, omega, faces)
    return Problem(name, n, h, tuple(src), omega, kappa, gamma, None, faces,
                   {"layer_cells": used, "ppw": ppw, "v0": v0, "grad": grad})


def linear_velocity_traveltime(n, h, src, v0, grad):
    """First-arrival time in v = v0 + grad*depth (textbook closed form).

    tau = arccosh(1 + grad^2 |x - x0|^2 / (2 v(x) v(x0))) / grad.  Used only
    to make test inputs and to check travel-time solvers; returns tau1 =
    tau / |x - x0| (tau1 at the source = 1 / v(x0)).
    """
    coords = node_coordinates(n, h)
    x0 = [s * hv for s, hv in zip(src, h)]
    r2 = sum((c - c0) ** 2 for c, c0 in zip(coords, x0))
    v = v0 + grad * coords[-1]
    vs = v0 + grad * x0[-1]
    tau = np.arccosh(1.0 + grad * grad * r2 / (2.0 * v * vs)) / grad
    r = np.sqrt(r2)
    tau1 = np.empty_like(tau)
    at_src = r == 0.0
    tau1[~at_src] = tau[~at_src] / r[~at_src]
    tau1[at_src] = 1.0 / vs
    return tau1


def smooth_random_field(n, seed, scale=0.1, modes=3):
    """Smooth seeded field 1 + scale * sum of low-frequency cosines (test inputs)."""
    rng = np.random.default_rng(seed)
    idx = node_coordinates(n, tuple(1.0 / max(v - 1, 1) for v in n))
    f = np.ones_like(idx[0])
    for _ in range(modes):
        k = rng.uniform(0.5, 2.0, size=len(n))
        ph = rng.uniform(0, 2 * math.pi, size=len(n))
        term = np.ones_like(idx[0])
        for d in range(len(n)):
            term = term * np.cos(math.pi * k[d] * idx[d] + ph[d])
        f = f + scale / modes * term
    return f


def random_complex(N, seed, dtype=np.complex128):
    """Seeded complex vector with standard-normal parts."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(dtype)


def batch_sources(n, count, seed=3, depth_layers=2):
    """Seeded surface source positions (lateral uniform, depth index < depth_layers)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        pos = [int(rng.integers(0, v)) for v in n[:-1]]
        pos.append(int(rng.integers(0, depth_layers)))
        out.append(tuple(pos))
    return out
