"""Batched operators: B problems on one grid (own source, frequency, slowness,
travel time and absorbing profile) in single launches.

The batch runs every problem with the same kernels, launch shapes and
reduction orders as a single-problem operator, so each problem's results
must be bit-for-bit those of its own single-problem operator: operator
applies, one cycle, the coefficients and Galerkin stencils, and whole solves
(iterates, per-problem iteration counts, residuals) in which the problems
converge at different iterations and are frozen in lockstep.
"""
import numpy as np
import pytest

from oracle import adr, eikonal
from paper_1712_06091_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _problems(kind):
    """List of (n, h, src, omega, kappa, tau1, gamma)."""
    if kind == "marine2d_65":
        base = W.marine_2d((65, 65))
        srcs = [base.src, (10, 1), (50, 3)]
        scales = [1.0, 0.8, 1.15]
        faces = base.layer_faces
    elif kind == "layered3d_17":
        base = W.layered_3d((17, 17, 9))
        srcs = [base.src, (3, 12, 1)]
        scales = [1.0, 0.9]
        faces = base.layer_faces
    else:  # ragged constant medium, sources on faces / corners
        base = W.constant_medium((17, 13, 9), src=(8, 6, 1))
        srcs = [(8, 6, 1), (0, 0, 0), (16, 12, 8)]
        scales = [1.0, 1.1, 0.7]
        faces = base.layer_faces
    g = adr.Grid(base.n, base.h)
    out = []
    for p, (s, sc) in enumerate(zip(srcs, scales)):
        kappa = base.kappa * (1.0 + 0.03 * p * (W.smooth_random_field(base.n, seed=20 + p) - 1.0))
        omega = base.omega * sc
        gamma, _ = W.absorbing_layer(base.n, base.h, kappa, omega, faces)
        tau1 = eikonal.factored_fast_marching(g, kappa, s, order=2)
        out.append((base.n, base.h, s, omega, kappa, tau1, gamma))
    return out


def _operators(kind, **overrides):
    from paper_1712_06091_gb300 import adr as gpu
    probs = _problems(kind)
    params = gpu.default_params(**overrides)
    n, h = probs[0][0], probs[0][1]
    stack = lambda k: torch.from_numpy(np.stack([p[k] for p in probs]))
    batch = gpu.BatchOperator(n, h, [p[2] for p in probs], [p[3] for p in probs], stack(4), stack(5), stack(6),
                              params=gpu.default_params(**overrides))
    singles = [gpu.Operator(n, h, p[2], p[3], torch.from_numpy(p[4]), torch.from_numpy(p[5]), torch.from_numpy(p[6]),
                            params=params) for p in probs]
    return probs, batch, singles


KINDS = ["marine2d_65", "layered3d_17", "ragged3d_17x13x9"]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_solve_equals_single_solves(adrlib, cuda, kind, precision):
    probs, batch, singles = _operators(kind, precision=precision, levels=3)
    tol = 1e-10 if precision == "f64" else 1e-8
    a, infos = batch.solve(tol=tol, maxit=400)
    a = a.reshape(len(probs), -1)
    for p, op in enumerate(singles):
        ap, info = op.solve(tol=tol, maxit=400)
        assert infos[p]["iterations"] == info["iterations"], (p, infos[p], info)
        assert infos[p]["rel_residual"] == info["rel_residual"]
        assert torch.equal(a[p], ap), p
    assert len({i["iterations"] for i in infos}) >= 1


@pytest.mark.parametrize("kind", KINDS)
def test_batch_operators_equal_single_operators(adrlib, cuda, kind):
    probs, batch, singles = _operators(kind, precision="f32", levels=3)
    B, N = len(probs), batch.nodes
    x = torch.from_numpy(np.stack([W.random_complex(N, 40 + p) for p in range(B)])).cuda()
    assert torch.equal(batch.apply(x.reshape(-1)).reshape(B, N), torch.stack([s.apply(x[p]) for p, s in enumerate(singles)]))
    x32 = x.to(torch.complex64)
    assert torch.equal(batch.apply(x32.reshape(-1), "prec").reshape(B, N),
                       torch.stack([s.apply(x32[p], "prec") for p, s in enumerate(singles)]))
    assert torch.equal(batch.vcycle(x32.reshape(-1)).reshape(B, N),
                       torch.stack([s.vcycle(x32[p]) for p, s in enumerate(singles)]))
    assert torch.equal(batch.coefficients(), torch.stack([s.coefficients() for s in singles]))
    for level in range(1, batch.info()["levels"].__len__()):
        assert torch.equal(batch.level_stencil(level), torch.stack([s.level_stencil(level) for s in singles]))
    q = batch.point_source_rhs().reshape(B, N)
    assert torch.equal(q, torch.stack([s.point_source_rhs() for s in singles]))
    u = batch.reconstruct(x.reshape(-1)).reshape(B, N)
    assert torch.equal(u, torch.stack([s.reconstruct(x[p]) for p, s in enumerate(singles)]))
    assert batch.info()["problems"] == B


def test_batch_update_and_refusals(adrlib, cuda):
    from paper_1712_06091_gb300 import _lib as L
    from paper_1712_06091_gb300 import adr as gpu
    probs, batch, singles = _operators("marine2d_65", precision="f32", levels=3)
    # swap the problems' order through an update: results follow the problems
    order = [2, 0, 1]
    stack = lambda k: torch.from_numpy(np.stack([probs[i][k] for i in order]))
    batch.update([probs[i][2] for i in order], [probs[i][3] for i in order], stack(4), stack(5), stack(6))
    a, infos = batch.solve(tol=1e-8)
    a = a.reshape(3, -1)
    for slot, i in enumerate(order):
        ai, info = singles[i].solve(tol=1e-8)
        assert torch.equal(a[slot], ai) and infos[slot]["iterations"] == info["iterations"]
    dummy = L.ctypes.c_void_p(16)   # never dereferenced: the batch is refused first
    rc = adrlib.adr_operator_update(batch._h, (L.ctypes.c_int * 3)(1, 1, 0), 1.0, dummy, dummy, dummy)
    assert rc == L.ADR_ERR_STATE
    n, h = probs[0][0], probs[0][1]
    with pytest.raises(L.ADRError):
        gpu.BatchOperator(n, h, [probs[0][2]] * 2, [probs[0][3]] * 2, np.stack([probs[0][4]] * 2),
                          np.stack([probs[0][5]] * 2), np.stack([probs[0][6]] * 2), params=gpu.default_params(adjoint=1))


def test_autotune_and_packed_solver(adrlib, cuda):
    """The tuner measures every candidate and the packed solve returns each
    problem's single-operator solution whatever the packing."""
    from paper_1712_06091_gb300 import adr as gpu
    from paper_1712_06091_gb300 import autotune
    probs = _problems("marine2d_65")
    n, h = probs[0][0], probs[0][1]
    problems = [(p[2], p[3], torch.from_numpy(p[4]).cuda(), torch.from_numpy(p[5]).cuda(), torch.from_numpy(p[6]).cuda())
                for p in probs]
    params = gpu.default_params(precision="f32", levels=3)
    tuned = autotune.tune(n, h, problems, params=params, packings=(1, 2, 3), relax_blocks=(8, 64))
    assert tuned["packing"] in (1, 2, 3) and tuned["relax_blocks"] in (8, 64)
    assert len(tuned["table"]) == 4 and all(r["ms_per_problem_iteration"] > 0 for r in tuned["table"])
    for packing in (2, 3):
        solver = autotune.PackedSolver(n, h, packing, params=params)
        us, infos = solver.solve(problems, tol=1e-8)
        solver.close()
        for p, (src, omega, kappa, tau1, gamma) in enumerate(problems):
            op = gpu.Operator(n, h, src, omega, kappa, tau1, gamma, params=params)
            a, info = op.solve(tol=1e-8)
            assert torch.equal(us[p], op.reconstruct(a)) and infos[p]["iterations"] == info["iterations"]


@pytest.mark.parametrize("form", ["grid", "cluster", "cta", "kernels"])
def test_batch_coarse_forms_equal_single(adrlib, cuda, form):
    probs, batch, singles = _operators("marine2d_65", precision="f32", levels=2, coarse_solver=form)
    a, infos = batch.solve(tol=1e-8)
    a = a.reshape(len(probs), -1)
    for p, op in enumerate(singles):
        ap, info = op.solve(tol=1e-8)
        assert torch.equal(a[p], ap) and infos[p]["iterations"] == info["iterations"], (form, p)
