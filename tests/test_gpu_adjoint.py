"""Adjoint path on the GPU against the oracle (conjugate-transposed CSR
matrices and hierarchies built by the oracle itself), the dot-product test,
and the slowness gradient against the oracle's and against central finite
differences of the GPU misfit (65 x 65, 4 sources).

Tolerances as in test_gpu_parity.py: single applications 1e-12, one cycle
and fixed-count FGMRES iterates 1e-10 relative L2; dot-product identity 1e-13.
Gradients: 1e-8 relative against the oracle (both solves to 1e-12) and 1e-6
against central differences with steps of 1e-6 |kappa|.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import adjoint as oadj
from oracle import adr, eikonal, krylov
from oracle import multigrid as mg
from paper_1712_06091_gb300 import workloads as W

from gpu_cases import CASES, make_operator, oracle_cycle_params, oracle_matrix, problem, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _cvec(x, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


def _hier_adjoint(name, params):
    P = problem(name)
    return mg.build_hierarchy(oracle_matrix(name, "prec").conj().T.tocsr(), P.n, params.levels)


@pytest.mark.parametrize("name", list(CASES))
def test_apply_adjoint_and_dot_product(adrlib, cuda, name):
    P, _, op = make_operator(name, precision="f64", adjoint=1)
    A = oracle_matrix(name, "2up")
    x = W.random_complex(P.N, 21)
    y = W.random_complex(P.N, 22)
    ahy = op.apply_adjoint(_cvec(y)).cpu().numpy()
    assert rel(ahy, A.conj().T @ y) <= 1e-12
    ax = op.apply(_cvec(x)).cpu().numpy()
    lhs, rhs = np.vdot(y, ax), np.vdot(ahy, x)     # <A x, y> = <x, A^H y>
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(ax) * np.linalg.norm(y)


CYCLES = [dict(), dict(cycle="V", relax="jacobi", sweeps=[1, 1, 1], jacobi_weight=[0.6] * 8)]


@pytest.mark.parametrize("name", ["const2d_33", "ragged2d_37x21", "marine2d_65", "layered3d_17", "corner3d_9x11x13"])
@pytest.mark.parametrize("ci", range(len(CYCLES)))
def test_adjoint_cycle_f64(adrlib, cuda, name, ci):
    P, params, op = make_operator(name, precision="f64", adjoint=1, **CYCLES[ci])
    hier = _hier_adjoint(name, params)
    r = W.random_complex(P.N, 23)
    z = op.vcycle_adjoint(_cvec(r)).cpu().numpy()
    ref = mg.cycle(hier, r, oracle_cycle_params(params))
    assert rel(z, ref) <= 1e-10, rel(z, ref)
    # the forward cycle on the same operator is untouched by the adjoint hierarchy
    hf = mg.build_hierarchy(oracle_matrix(name, "prec"), P.n, params.levels)
    zf = op.vcycle(_cvec(r)).cpu().numpy()
    assert rel(zf, mg.cycle(hf, r, oracle_cycle_params(params))) <= 1e-10


@pytest.mark.parametrize("name", ["const2d_33", "marine2d_65", "layered3d_17"])
def test_adjoint_cycle_f32(adrlib, cuda, name):
    P, params, op = make_operator(name, precision="f32", adjoint=1)
    hier = _hier_adjoint(name, params)
    r = W.random_complex(P.N, 24)
    z = op.vcycle_adjoint(_cvec(r, torch.complex64)).cpu().numpy()
    assert rel(z, mg.cycle(hier, r, oracle_cycle_params(params))) <= 2e-4


@pytest.mark.parametrize("name", ["const2d_33", "marine2d_65", "layered3d_17"])
def test_adjoint_fgmres_iterates(adrlib, cuda, name):
    k, m = 7, 4
    P, params, op = make_operator(name, precision="f64", adjoint=1, restart=m)
    AH = oracle_matrix(name, "2up").conj().T.tocsr()
    hier = _hier_adjoint(name, params)
    prm = oracle_cycle_params(params)
    f = W.random_complex(P.N, 25)
    x_ref, its, res, _ = krylov.fgmres(AH, f, lambda v: mg.cycle(hier, v, prm), tol=0.0, restart=m, maxit=k,
                                       reorth_eta=params.reorth_eta)
    lam, info = op.adjoint_solve(_cvec(f), tol=0.0, maxit=k, raise_on_fail=False)
    assert info["iterations"] == its == k
    assert rel(lam.cpu().numpy(), x_ref) <= 1e-10


@pytest.mark.parametrize("name", ["ragged2d_37x21", "const3d_17x13x9", "layered3d_17"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_adjoint_solve_to_direct(adrlib, cuda, name, precision):
    P, _, op = make_operator(name, precision=precision, adjoint=1)
    AH = oracle_matrix(name, "2up").conj().T.tocsc()
    f = W.random_complex(P.N, 26)
    lam, info = op.adjoint_solve(_cvec(f), tol=1e-12, maxit=400)
    assert info["rel_residual"] <= 1e-12
    assert rel(lam.cpu().numpy(), spla.spsolve(AH, f)) <= 1e-9


def test_adjoint_requires_the_flag(adrlib, cuda):
    from paper_1712_06091_gb300 import _lib as L
    P, _, op = make_operator("const2d_33")
    x = _cvec(W.random_complex(P.N, 1))
    with pytest.raises(L.ADRError) as e:
        op.apply_adjoint(x)
    assert e.value.code == L.ADR_ERR_STATE


def _gradient_problem(n, nsrc, seed):
    P = W.marine_2d(n)
    g = adr.Grid(P.n, P.h)
    rng = np.random.default_rng(seed)
    sources = [(int(x), 1) for x in rng.choice(np.arange(4, n[0] - 4), size=nsrc, replace=False)]
    tau1s = [eikonal.factored_fast_marching(g, P.kappa, s, order=2) for s in sources]
    rec = np.arange(2, n[0] - 2, 2, dtype=np.int64)       # surface line
    kappa_true = P.kappa * (1.0 + 0.02 * W.smooth_random_field(P.n, seed=11))
    data = [oadj.forward_wavefield(g, s, P.omega, kappa_true, P.gamma, t1)[2][rec] for s, t1 in zip(sources, tau1s)]
    return P, g, sources, tau1s, rec, data


def test_gradient_matches_oracle(adrlib, cuda):
    from paper_1712_06091_gb300 import adr as gpu
    P, g, sources, tau1s, rec, data = _gradient_problem((33, 33), 2, 5)
    J_ref, g_ref = oadj.misfit_gradient(g, sources, P.omega, P.kappa, P.gamma, tau1s, rec, data)
    params = gpu.default_params(precision="f64")
    J, grad = gpu.misfit_gradient(P.n, P.h, P.omega, P.kappa, P.gamma, sources, tau1s, torch.from_numpy(rec).cuda(),
                                  [_cvec(d) for d in data], params=params, tol=1e-12)
    assert abs(J - J_ref) <= 1e-9 * J_ref
    assert rel(grad.cpu().numpy(), g_ref) <= 1e-8


def test_gradient_central_differences_65x65_four_sources(adrlib, cuda):
    """FP64 outer / FP32 preconditioner; directional derivatives on 20 random node subsets."""
    from paper_1712_06091_gb300 import adr as gpu
    P, g, sources, tau1s, rec, data = _gradient_problem((65, 65), 4, 9)
    rec_t = torch.from_numpy(rec).cuda()
    data_t = [_cvec(d) for d in data]
    kw = dict(n=P.n, h=P.h, omega=P.omega, gamma=P.gamma, sources=sources, tau1s=tau1s, receivers=rec_t,
              data=data_t, tol=1e-13, maxit=600)
    kappa = torch.from_numpy(P.kappa).cuda()
    J, grad = gpu.misfit_gradient(kappa=kappa, **kw)
    grad = grad.cpu().numpy()
    rng = np.random.default_rng(13)
    worst = 0.0
    for trial in range(20):
        v = np.zeros(P.N)
        subset = rng.choice(P.N, size=P.N // 16, replace=False)
        v[subset] = rng.standard_normal(subset.size) * P.kappa[subset]
        eps = 1e-6
        vt = torch.from_numpy(v).cuda()
        Jp, _ = gpu.misfit_gradient(kappa=kappa + eps * vt, **kw)
        Jm, _ = gpu.misfit_gradient(kappa=kappa - eps * vt, **kw)
        fd = (Jp - Jm) / (2 * eps)
        an = float(grad @ v)
        worst = max(worst, abs(fd - an) / abs(an))
    assert worst <= 1e-6, worst


def test_autograd_function(adrlib, cuda):
    from paper_1712_06091_gb300 import adr as gpu
    P, g, sources, tau1s, rec, data = _gradient_problem((33, 33), 2, 5)
    problem_kw = dict(n=P.n, h=P.h, omega=P.omega, gamma=P.gamma, sources=sources, tau1s=tau1s,
                      receivers=torch.from_numpy(rec).cuda(), data=[_cvec(d) for d in data], tol=1e-12)
    kappa = torch.from_numpy(P.kappa).cuda().requires_grad_(True)
    J = gpu.KappaMisfit.apply(kappa, problem_kw)
    (2.0 * J).backward()
    J2, grad = gpu.misfit_gradient(kappa=kappa.detach(), **problem_kw)
    assert abs(float(J.detach()) - J2) <= 1e-12 * J2
    assert rel(kappa.grad.cpu().numpy(), 2.0 * grad.cpu().numpy()) <= 1e-12
