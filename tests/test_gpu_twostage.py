"""GPU two-stage central solve (Algorithm ADRlong) against the oracle, through the C ABI.

The library runs stage 2 on the amplitude with the preconditioner
M^{-1} K M (K the cycle on H_s^cen = M H_cen M^{-1} - i alpha w^2 kappa^2);
the oracle runs it on u = M a as the paper writes it.  M is unitary, so the
FGMRES iterates map onto each other exactly in exact arithmetic and agree to
the solver's float64 parity target (1e-10 relative) in practice.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import adr, krylov, twostage
from oracle import multigrid as mg
from paper_1712_06091_gb300 import workloads as W

from gpu_cases import oracle_cycle_params, problem, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NAMES = ["marine2d_65", "ragged2d_37x21", "layered3d_17", "corner3d_9x11x13"]


def _cvec(x, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


def _ops(name, **kw):
    from paper_1712_06091_gb300 import adr as gpu
    P = problem(name)
    p1, p2 = gpu.central_two_stage_params(**kw)
    args = (P.n, P.h, P.src, P.omega, torch.from_numpy(P.kappa), torch.from_numpy(P.tau1), torch.from_numpy(P.gamma))
    return P, gpu.Operator(*args, params=p1), gpu.Operator(*args, params=p2), p1, p2


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_rescaled_shifted_cycle_operator(adrlib, cuda, name, precision):
    P, op1, op2, _, _ = _ops(name, precision=precision)
    g = adr.Grid(P.n, P.h)
    Hs = twostage.shifted_rescaled_central(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, 0.2)
    x = W.random_complex(g.N, 23)
    dt = torch.complex128 if precision == "f64" else torch.complex64
    y = op2.apply(_cvec(x, dt), "prec").cpu().numpy()
    ref = Hs @ x
    assert np.abs(y - ref).max() / np.abs(ref).max() <= (1e-12 if precision == "f64" else 1e-5)
    # the outer operators: H_cen (stage 2) and H_1up (stage 1), the stage-1 cycle on H_1up
    for op, scheme in ((op2, "cen"), (op1, "1up")):
        y = op.apply(_cvec(x), scheme).cpu().numpy()
        A = adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, scheme)
        assert np.abs(y - A @ x).max() / np.abs(A @ x).max() <= 1e-12
    if precision == "f64":
        y = op1.apply(_cvec(x), "prec").cpu().numpy()
        A = adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, "1up")
        assert np.abs(y - A @ x).max() / np.abs(A @ x).max() <= 1e-12


@pytest.mark.parametrize("name", NAMES)
def test_rescaled_shifted_cycle_f64(adrlib, cuda, name):
    P, _, op2, _, p2 = _ops(name, precision="f64")
    g = adr.Grid(P.n, P.h)
    hier = mg.build_hierarchy(twostage.shifted_rescaled_central(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, 0.2),
                              P.n, p2.levels)
    r = W.random_complex(g.N, 29)
    z = op2.vcycle(_cvec(r)).cpu().numpy()
    assert rel(z, mg.cycle(hier, r, oracle_cycle_params(p2))) <= 1e-10


@pytest.mark.parametrize("name", ["marine2d_65", "layered3d_17", "corner3d_9x11x13"])
def test_stage2_iterates_match_rescaled_oracle(adrlib, cuda, name):
    """Fixed-count stage-2 FGMRES from zero: the library's amplitude iterate
    equals M^{-1} times the oracle's u-space iterate."""
    P, _, op2, _, p2 = _ops(name, precision="f64", restart=5)
    g = adr.Grid(P.n, P.h)
    m = twostage.phase(g, P.src, P.omega, P.tau1)
    A2 = twostage.rescaled(adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, "cen"), m)
    hier = mg.build_hierarchy(twostage.shifted_rescaled_central(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, 0.2),
                              P.n, p2.levels)
    q = m * adr.point_source_rhs(g, P.src)
    u_ref, its, res, _ = krylov.fgmres(A2, q, lambda v: mg.cycle(hier, v, oracle_cycle_params(p2)), tol=0.0,
                                       restart=5, maxit=7, reorth_eta=p2.reorth_eta)
    a, info = op2.solve(tol=0.0, maxit=7, raise_on_fail=False)
    assert info["iterations"] == its == 7
    assert rel(a.cpu().numpy(), u_ref / m) <= 1e-10
    assert abs(info["rel_residual"] - res) <= 1e-8 * res


@pytest.mark.parametrize("name", ["marine2d_65", "layered3d_17"])
def test_two_stage_matches_oracle(adrlib, cuda, name):
    """Both stages with the paper's stage-1 rule (1e-2 or 5 iterations) and a
    fixed stage-2 count: iterate parity with the oracle's Algorithm ADRlong."""
    from paper_1712_06091_gb300 import adr as gpu
    P, op1, op2, p1, p2 = _ops(name, precision="f64", restart=5)
    g = adr.Grid(P.n, P.h)
    u_ref, a_ref, (its1, res1), (its2, res2) = twostage.two_stage_central(
        g, P.src, P.omega, P.kappa, P.gamma, P.tau1, oracle_cycle_params(p2), p2.levels, alpha=0.2, tol=0.0,
        restart=5, maxit=6, reorth_eta=p2.reorth_eta)
    a, i1, i2 = gpu.solve_two_stage(op1, op2, tol1=1e-2, maxit1=5, tol=0.0, maxit=6, raise_on_fail=False)
    assert i1[0]["iterations"] == its1 and i2[0]["iterations"] == its2 == 6
    assert abs(i1[0]["rel_residual"] - res1) <= 1e-8 * res1
    assert rel(a.cpu().numpy(), a_ref) <= 1e-10


@pytest.mark.parametrize("name", ["marine2d_65", "const3d_17x13x9", "layered3d_17"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_two_stage_solves_central_system(adrlib, cuda, name, precision):
    """float32 or float64 cycles: the float64 residual of H_cen a = q_hat
    reaches 1e-8 and a matches the direct solution."""
    from paper_1712_06091_gb300 import adr as gpu
    P, op1, op2, _, _ = _ops(name, precision=precision)
    g = adr.Grid(P.n, P.h)
    a, i1, i2 = gpu.solve_two_stage(op1, op2, tol=1e-8, maxit=600)
    a = a.cpu().numpy()
    Ac = adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, "cen")
    q = adr.point_source_rhs(g, P.src)
    true_res = np.linalg.norm(q - Ac @ a) / np.linalg.norm(q)
    assert true_res <= 1.0000001e-8 and abs(true_res - i2[0]["rel_residual"]) <= 1e-12
    assert i1[0]["iterations"] <= 5
    assert rel(a, spla.spsolve(Ac.tocsc(), q)) <= 1e-4


def test_two_stage_batch_matches_single(adrlib, cuda):
    """Two problems (own source and frequency) in one batched pair of
    operators: each problem's result equals its own single-problem solve."""
    from paper_1712_06091_gb300 import adr as gpu
    P = problem("layered3d_17")
    srcs = [P.src, (4, 5, 1)]
    omegas = [P.omega, 0.8 * P.omega]
    kap = torch.from_numpy(np.concatenate([P.kappa, P.kappa]))
    gam = torch.from_numpy(np.concatenate([P.gamma, P.gamma]))
    from oracle import eikonal
    taus = [P.tau1, eikonal.factored_fast_marching(adr.Grid(P.n, P.h), P.kappa, srcs[1], order=2)]
    tau = torch.from_numpy(np.concatenate(taus))
    p1, p2 = gpu.central_two_stage_params(precision="f64")
    b1 = gpu.BatchOperator(P.n, P.h, srcs, omegas, kap, tau, gam, params=p1)
    b2 = gpu.BatchOperator(P.n, P.h, srcs, omegas, kap, tau, gam, params=p2)
    a, i1, i2 = gpu.solve_two_stage(b1, b2, tol=1e-10, maxit=400)
    N = P.N
    for k in range(2):
        args = (P.n, P.h, srcs[k], omegas[k], torch.from_numpy(P.kappa), torch.from_numpy(taus[k]),
                torch.from_numpy(P.gamma))
        s1, s2 = gpu.Operator(*args, params=p1), gpu.Operator(*args, params=p2)
        ak, j1, j2 = gpu.solve_two_stage(s1, s2, tol=1e-10, maxit=400)
        assert i1[k]["iterations"] == j1[0]["iterations"]
        assert rel(a[k * N:(k + 1) * N].cpu().numpy(), ak.cpu().numpy()) <= 1e-8


def test_two_stage_argument_errors(adrlib, cuda):
    from paper_1712_06091_gb300 import _lib as L
    from paper_1712_06091_gb300 import adr as gpu
    P, op1, op2, _, _ = _ops("const3d_17x13x9", precision="f64")
    Q = problem("layered3d_17")
    other = gpu.Operator(Q.n, Q.h, Q.src, Q.omega, torch.from_numpy(Q.kappa), torch.from_numpy(Q.tau1),
                         torch.from_numpy(Q.gamma))
    with pytest.raises(L.ADRError):
        gpu.solve_two_stage(op1, other)
    with pytest.raises(L.ADRError):
        gpu.solve_two_stage(op1, op1)
