"""Shared GPU-test helpers: seeded problems, their oracle matrices, and the
conversion of library parameters to the oracle's cycle settings."""
import copy
import functools

import numpy as np

from oracle import adr, eikonal
from oracle import multigrid as mg
from paper_1712_06091_gb300 import workloads as W

# (name, builder): sizes span several 256-thread tiles with ragged tails,
# 2D and 3D, anisotropic spacing, sources in the interior, on a face and at a
# corner-adjacent node, constant and heterogeneous media.
CASES = {
    "const2d_33": lambda: W.constant_medium((33, 33)),
    "ragged2d_37x21": lambda: W.constant_medium((37, 21), extent=1.0, src=(2, 0), faces=W.faces_except_surface(2)),
    "marine2d_65": lambda: _with_fm(W.marine_2d((65, 65))),
    "const3d_17x13x9": lambda: W.constant_medium((17, 13, 9), src=(8, 6, 1)),
    "layered3d_17": lambda: _with_fm(W.layered_3d((17, 17, 9))),
    "corner3d_9x11x13": lambda: W.constant_medium((9, 11, 13), src=(1, 0, 0)),
    # level 1 = 25 x 25 x 13 = 8125 nodes = 254 tiles of 32: with a grid of one or
    # two blocks every warp of the streamed relaxation walks 8 to 32 tiles
    "const3d_49x49x25": lambda: W.constant_medium((49, 49, 25), src=(24, 24, 2), faces=W.faces_except_surface(3)),
}


def _with_fm(P):
    g = adr.Grid(P.n, P.h)
    P.tau1 = eikonal.factored_fast_marching(g, P.kappa, P.src, order=2)
    return P


@functools.lru_cache(maxsize=None)
def problem(name):
    """A case by name; the suffix ":helmholtz" gives the same medium and source
    with tau1 = 0, i.e. the standard Helmholtz matrix (Sec. 1)."""
    if name.endswith(":helmholtz"):
        P = copy.copy(problem(name[: -len(":helmholtz")]))
        P.tau1 = np.zeros_like(P.tau1)
        return P
    return CASES[name]()


@functools.lru_cache(maxsize=None)
def oracle_matrix(name, scheme, near=1, beta=0.25, shift=0.0):
    P = problem(name)
    g = adr.Grid(P.n, P.h)
    if scheme == "prec":
        return adr.assemble_preconditioner(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, beta, near, shift)
    return adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, scheme, near)


def oracle_cycle_params(p):
    return mg.CycleParams(cycle="VK"[p.cycle], relax=["jacobi", "mr"][p.relax], pre=list(p.pre_sweeps),
                          post=list(p.post_sweeps), weights=list(p.jacobi_weight),
                          coarse_iterations=p.coarse_iterations, kcycle_iterations=p.kcycle_iterations,
                          kcycle_threshold=p.kcycle_threshold,
                          coarse_reorth_eta=p.reorth_eta if p.reorth_eta < 1.0 else None)


def make_operator(name, **overrides):
    import torch
    from paper_1712_06091_gb300 import adr as gpu
    P = problem(name)
    params = gpu.default_params(**overrides)
    op = gpu.Operator(P.n, P.h, P.src, P.omega, torch.from_numpy(P.kappa), torch.from_numpy(P.tau1),
                      torch.from_numpy(P.gamma), params=params)
    return P, params, op


def pattern_offsets(dim):
    out = []
    if dim == 2:
        for o1 in range(-2, 3):
            for o0 in range(-2, 3):
                if (abs(o0) == 2) + (abs(o1) == 2) <= 1:
                    out.append((o0, o1))
    else:
        for o2 in range(-2, 3):
            for o1 in range(-2, 3):
                for o0 in range(-2, 3):
                    if (abs(o0) == 2) + (abs(o1) == 2) + (abs(o2) == 2) <= 1:
                        out.append((o0, o1, o2))
    return out


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)
