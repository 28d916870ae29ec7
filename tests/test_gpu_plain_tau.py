"""adr_operator_create_tau (a travel time given as plain nodal values, its
derivatives by finite differences) against the oracle assembled from the same
plain tau (oracle.adr.PlainTau), element by element through the C ABI.

Tolerances as in test_gpu_parity: 1e-12 for coefficients and single float64
applications, 1e-10 for one float64 cycle, solves against the direct
solution of the same matrix to 1e-10 / 1e-8."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import adr
from oracle import multigrid as mg
from paper_1712_06091_gb300 import workloads as W

from gpu_cases import oracle_cycle_params, problem, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NAMES = ["marine2d_65", "layered3d_17", "corner3d_9x11x13"]


def _plain(name):
    """The case's travel time tau = |x - x0| tau1 as plain values (a
    plain-tau input a user would have from any eikonal solver)."""
    P = problem(name)
    g = adr.Grid(P.n, P.h)
    return P, g, adr.travel_time(g, P.src, P.tau1)


def _operator(P, tau, **kw):
    from paper_1712_06091_gb300 import adr as gpu
    params = gpu.default_params(**kw)
    return params, gpu.Operator(P.n, P.h, P.src, P.omega, torch.from_numpy(P.kappa), torch.from_numpy(tau),
                                torch.from_numpy(P.gamma), params=params, tau_kind="plain")


@pytest.mark.parametrize("name", NAMES)
def test_plain_tau_coefficients_and_apply(adrlib, cuda, name):
    P, g, tau = _plain(name)
    _, op = _operator(P, tau, precision="f64")
    got = op.coefficients().cpu().numpy()
    D = len(P.n)
    T = adr.PlainTau(tau)
    js = g.index(P.src)
    for j in range(g.N):
        tv, gr, t, rho = adr.node_coefficients(g, P.src, P.omega, P.kappa, P.gamma, T, j)
        if j == js:
            continue
        ref = list(gr) + list(t) + [rho.real, rho.imag, tv]
        for k, v in enumerate(ref):
            scale = P.omega ** 2 * P.kappa.max() ** 2 if k == 2 * D else max(1.0, abs(v))
            assert abs(got[k, j] - v) <= 1e-11 * scale, (name, j, k, got[k, j], v)
    x = W.random_complex(g.N, 21)
    xd = torch.from_numpy(x).cuda()
    for scheme in ("2up", "1up", "cen"):
        A = adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, T, scheme)
        y = op.apply(xd, scheme).cpu().numpy()
        assert rel(y, A @ x) <= 1e-12, (name, scheme, rel(y, A @ x))


@pytest.mark.parametrize("name", NAMES)
def test_plain_tau_cycle_and_solve(adrlib, cuda, name):
    P, g, tau = _plain(name)
    T = adr.PlainTau(tau)
    params, op = _operator(P, tau, precision="f64", levels=3)
    hier = mg.build_hierarchy(adr.assemble_preconditioner(g, P.src, P.omega, P.kappa, P.gamma, T), P.n, params.levels)
    r = W.random_complex(g.N, 22)
    z = op.vcycle(torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel(z, mg.cycle(hier, r, oracle_cycle_params(params))) <= 1e-10
    A = adr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, T, "2up")
    q = adr.point_source_rhs(g, P.src)
    xe = spla.spsolve(A.tocsc(), q)
    a, info = op.solve(tol=1e-12, maxit=400)
    assert info["rel_residual"] <= 1e-12 and rel(a.cpu().numpy(), xe) <= 1e-10
    u = op.reconstruct(a).cpu().numpy()
    assert rel(u, adr.reconstruct(g, P.src, P.omega, T, xe)) <= 1e-10
    # the float32 cycle inside the float64 iteration reaches 1e-8
    _, op32 = _operator(P, tau, precision="f32", levels=3)
    a32, info32 = op32.solve(tol=1e-8, maxit=400)
    res = np.linalg.norm(q - A @ a32.cpu().numpy()) / np.linalg.norm(q)
    assert info32["rel_residual"] <= 1e-8 and res <= 1.0000001e-8
