"""Batches of problems with grids of their own (adr_batch_create_grids): the
many-frequency setting, each frequency on the coarsest grid that keeps its
points per wavelength, every problem of every size in one launch per step.

Each problem's arithmetic is that of its own single-problem operator; only
the block partitioning of reductions follows the batch's largest grid, so
results agree to rounding: one float64 cycle and fixed-count float64 FGMRES
iterates to 1e-12 / 1e-10, float64 solves to 1e-12 against the oracle's
direct solution, float32-cycle solves to 1e-8 with the single problem's
iteration count (within one) and its solution (to the solve's accuracy).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import adr, eikonal
from paper_1712_06091_gb300 import workloads as W

from gpu_cases import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _problems(dim):
    """(n, h, src, omega, kappa, tau1, gamma) per problem: the same model family
    resampled to three grids, the frequency scaled with the resolution (10
    points per wavelength on each)."""
    if dim == 2:
        shapes = [(33, 33), (65, 65), (49, 33)]
        build = lambda n: W.marine_2d(n)
    else:
        shapes = [(17, 17, 9), (33, 33, 17), (25, 25, 13)]
        build = lambda n: W.layered_3d(n)
    out = []
    for k, n in enumerate(shapes):
        P = build(n)
        g = adr.Grid(P.n, P.h)
        src = tuple(min(s + k, v - 1) for s, v in zip(P.src, P.n))
        tau1 = eikonal.factored_fast_marching(g, P.kappa, src, order=2)
        out.append((P.n, P.h, src, P.omega, P.kappa, tau1, P.gamma))
    return out


def _operators(dim, **kw):
    from paper_1712_06091_gb300 import adr as gpu
    probs = _problems(dim)
    cat = lambda k: torch.from_numpy(np.concatenate([p[k] for p in probs]))
    batch = gpu.GridsBatchOperator([(p[0], p[1]) for p in probs], [p[2] for p in probs], [p[3] for p in probs],
                                   cat(4), cat(5), cat(6), params=gpu.default_params(**kw))
    singles = [gpu.Operator(p[0], p[1], p[2], p[3], torch.from_numpy(p[4]), torch.from_numpy(p[5]),
                            torch.from_numpy(p[6]), params=gpu.default_params(**kw)) for p in probs]
    return probs, batch, singles


@pytest.mark.parametrize("dim", [2, 3])
def test_grids_batch_layout_and_coefficients(adrlib, cuda, dim):
    probs, batch, singles = _operators(dim, precision="f64", levels=3)
    assert batch.N == sum(int(np.prod(p[0])) for p in probs)
    assert batch.info()["problems"] == 3 and len(batch.info()["levels"]) == 3
    co = batch.coefficients()
    off = 0
    for p, op in enumerate(singles):
        c = op.coefficients().reshape(-1)
        assert torch.equal(co[off:off + c.numel()], c), p   # elementwise setup: identical
        off += c.numel()


@pytest.mark.parametrize("dim", [2, 3])
def test_grids_batch_cycle_and_iterates_f64(adrlib, cuda, dim):
    probs, batch, singles = _operators(dim, precision="f64", levels=3)
    r = torch.from_numpy(W.random_complex(batch.N, 31)).cuda()
    zb = batch.split(batch.vcycle(r))
    for p, (op, rp) in enumerate(zip(singles, batch.split(r))):
        z = op.vcycle(rp.clone())
        assert rel(zb[p].cpu().numpy(), z.cpu().numpy()) <= 1e-12, p
    ab, _ = batch.solve(tol=0.0, maxit=7, raise_on_fail=False)
    for p, (op, a) in enumerate(zip(singles, batch.split(ab))):
        a1, _ = op.solve(tol=0.0, maxit=7, raise_on_fail=False)
        assert rel(a.cpu().numpy(), a1.cpu().numpy()) <= 1e-10, p


def test_grids_batch_solve_f64_against_direct(adrlib, cuda):
    """Every problem of the 2D batch solved to 1e-12 with the float64 cycle
    equals the direct solution of its own oracle matrix."""
    probs, batch, _ = _operators(2, precision="f64", levels=3)
    ab, infos = batch.solve(tol=1e-12, maxit=600)
    for p, (pr, a) in enumerate(zip(probs, batch.split(ab))):
        n, h, src, omega, kappa, tau1, gamma = pr
        g = adr.Grid(n, h)
        A = adr.assemble_adr(g, src, omega, kappa, gamma, tau1, "2up")
        xe = spla.spsolve(A.tocsc(), adr.point_source_rhs(g, src))
        assert infos[p]["rel_residual"] <= 1e-12 and rel(a.cpu().numpy(), xe) <= 1e-9, (p, infos[p])


@pytest.mark.parametrize("dim", [2, 3])
def test_grids_batch_solve_f32(adrlib, cuda, dim):
    probs, batch, singles = _operators(dim, precision="f32", levels=3)
    ab, infos = batch.solve(tol=1e-8, maxit=600)
    ub = batch.split(batch.reconstruct(ab))
    for p, (op, a) in enumerate(zip(singles, batch.split(ab))):
        a1, info = op.solve(tol=1e-8, maxit=600)
        assert infos[p]["rel_residual"] <= 1e-8 and abs(infos[p]["iterations"] - info["iterations"]) <= 1, \
            (p, infos[p], info)
        assert rel(a.cpu().numpy(), a1.cpu().numpy()) <= 1e-6, p
        assert rel(ub[p].cpu().numpy(), op.reconstruct(a1).cpu().numpy()) <= 1e-6, p


def test_grids_batch_rejects_unequal_depth(adrlib, cuda):
    """The hierarchy stops where any problem stops; a problem whose grid cannot
    coarsen as far as the others' still builds (fewer levels for everyone)."""
    from paper_1712_06091_gb300 import adr as gpu
    n1, n2 = (33, 33), (9, 9)     # 9 -> 5 -> 3: three levels at most; 33 allows five
    P1, P2 = W.marine_2d(n1), W.marine_2d(n2)
    cat = lambda a, b: torch.from_numpy(np.concatenate([a, b]))
    op = gpu.GridsBatchOperator([(P1.n, P1.h), (P2.n, P2.h)], [P1.src, P2.src], [P1.omega, P2.omega],
                                cat(P1.kappa, P2.kappa), cat(P1.kappa, P2.kappa), cat(P1.gamma, P2.gamma),
                                params=gpu.default_params(levels=5))
    assert len(op.info()["levels"]) == 3
