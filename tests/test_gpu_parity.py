"""GPU path vs the oracle, element by element, through the C ABI.

Tolerances (float64 arithmetic, unit roundoff 1.1e-16):
  * coefficients and single operator applications: 1e-12 relative (a few
    dozen roundings of terms of equal sign; FMA contraction differs);
  * Galerkin stencils: 1e-12 relative to the largest entry of the level;
  * one multigrid cycle and fixed-count FGMRES iterates: 1e-10 relative L2
    (the solver's parity target; rounding differences are amplified by the
    Krylov recurrences and the nonlinear fixed-count coarse solves);
  * float32 applications: 1e-5 relative (unit roundoff 6e-8 times the
    cancellation between the Laplacian and the reaction terms).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import adr, krylov
from oracle import multigrid as mg
from paper_1712_06091_gb300 import workloads as W

from gpu_cases import CASES, make_operator, oracle_cycle_params, oracle_matrix, pattern_offsets, problem, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NAMES = list(CASES)


def _cvec(x, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


@pytest.mark.parametrize("name", NAMES)
def test_coefficients(adrlib, cuda, name):
    P, _, op = make_operator(name)
    got = op.coefficients().cpu().numpy()
    g = adr.Grid(P.n, P.h)
    D = len(P.n)
    ref = np.zeros_like(got)
    for j in range(g.N):
        tau, gr, t, rho = adr.node_coefficients(g, P.src, P.omega, P.kappa, P.gamma, P.tau1, j)
        ref[:D, j] = gr
        ref[D:2 * D, j] = t
        ref[2 * D, j] = rho.real
        ref[2 * D + 1, j] = rho.imag
        ref[2 * D + 2, j] = tau
    js = g.index(P.src)
    mask = np.ones(g.N, bool)
    mask[js] = False       # derivatives at the source are never used (its row is M^-1 H M)
    for k in range(got.shape[0]):
        scale = max(np.abs(ref[k, mask]).max(), 1e-300)
        if k == 2 * D:      # Re rho = w^2 (kappa^2 - |grad tau|^2) cancels: compare on the scale of w^2 kappa^2
            scale = P.omega ** 2 * np.max(P.kappa) ** 2
        assert np.abs(got[k, mask] - ref[k, mask]).max() <= 1e-12 * scale, (name, k)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("scheme", ["2up", "1up", "cen", "prec"])
def test_apply_f64(adrlib, cuda, name, scheme):
    P, _, op = make_operator(name)
    A = oracle_matrix(name, scheme)
    x = W.random_complex(A.shape[0], 7)
    y = op.apply(_cvec(x), scheme).cpu().numpy()
    ref = A @ x
    err = np.abs(y - ref).max() / np.abs(ref).max()
    assert err <= 1e-12, (name, scheme, err)


@pytest.mark.parametrize("name", ["const2d_33", "marine2d_65", "layered3d_17"])
def test_apply_f32(adrlib, cuda, name):
    P, _, op = make_operator(name)
    A = oracle_matrix(name, "2up")
    x = W.random_complex(A.shape[0], 8)
    y = op.apply(_cvec(x, torch.complex64), "2up").cpu().numpy()
    ref = A @ x
    assert np.abs(y - ref).max() / np.abs(ref).max() <= 1e-5


@pytest.mark.parametrize("near", [1, 2])
def test_apply_near_source_radius(adrlib, cuda, near):
    P, _, op = make_operator("marine2d_65", near_source=near)
    A = oracle_matrix("marine2d_65", "2up", near)
    x = W.random_complex(A.shape[0], 9)
    y = op.apply(_cvec(x), "2up").cpu().numpy()
    assert np.abs(y - A @ x).max() / np.abs(A @ x).max() <= 1e-12


@pytest.mark.parametrize("name", ["const2d_33", "ragged2d_37x21", "marine2d_65", "const3d_17x13x9", "layered3d_17"])
def test_galerkin_stencils(adrlib, cuda, name):
    P, params, op = make_operator(name, precision="f64")
    hier = mg.build_hierarchy(oracle_matrix(name, "prec"), P.n, params.levels)
    info = op.info()
    assert [lv["n"] for lv in info["levels"]] == [tuple(lv["n"]) for lv in hier]
    offs = pattern_offsets(len(P.n))
    for l in range(1, len(hier)):
        st = op.level_stencil(l).cpu().numpy()
        Ac = hier[l]["A"].tocsr()
        gc = adr.Grid(hier[l]["n"], (1.0,) * len(P.n))
        dense = np.zeros_like(st)
        for I in range(gc.N):
            ci = gc.coords(I)
            row = dict(zip(Ac[I].indices, Ac[I].data))
            seen = 0
            for p, o in enumerate(offs):
                cj = tuple(ci[d] + o[d] for d in range(len(o)))
                if gc.inside(cj):
                    J = gc.index(cj)
                    dense[p, I] = row.get(J, 0.0)
                    seen += J in row
            assert seen == len(row), "oracle entry outside the pattern"
        scale = np.abs(dense).max()
        assert np.abs(st - dense).max() <= 1e-12 * scale, (name, l)


CYCLES = [
    dict(),                                                   # K-cycle, MR relaxation, l+1 sweeps
    dict(cycle="V", levels=3),
    dict(cycle="V", relax="jacobi", sweeps=1, jacobi_weight=[0.6, 0.5, 0.4, 0.4, 0.4]),
    dict(levels=1, coarse_iterations=7),
    dict(kcycle_iterations=3, sweeps=[1, 2, 1], coarse_iterations=5),
]


@pytest.mark.parametrize("name", ["const2d_33", "ragged2d_37x21", "marine2d_65", "layered3d_17", "corner3d_9x11x13"])
@pytest.mark.parametrize("ci", range(len(CYCLES)))
def test_cycle_f64(adrlib, cuda, name, ci):
    P, params, op = make_operator(name, precision="f64", **CYCLES[ci])
    hier = mg.build_hierarchy(oracle_matrix(name, "prec"), P.n, params.levels)
    prm = oracle_cycle_params(params)
    r = W.random_complex(hier[0]["A"].shape[0], 11)
    z = op.vcycle(_cvec(r)).cpu().numpy()
    ref = mg.cycle(hier, r, prm)
    assert rel(z, ref) <= 1e-10, (name, ci, rel(z, ref))


@pytest.mark.parametrize("name", ["marine2d_65", "layered3d_17", "const3d_17x13x9"])
@pytest.mark.parametrize("threshold", [0.1, 0.6, 1.0])
def test_kcycle_early_exit_f64(adrlib, cuda, name, threshold):
    """Alg. Kcycle with the coarse threshold of Sec. 4.2: an inner FGMRES whose
    first step already reduces the residual to `threshold` of the restricted
    residual stops there (1.0 always stops; 0.1 and 0.6 depend on the level).
    One cycle, then fixed-count FGMRES iterates, against the oracle."""
    P, params, op = make_operator(name, precision="f64", levels=4, kcycle_threshold=threshold)
    hier = mg.build_hierarchy(oracle_matrix(name, "prec"), P.n, params.levels)
    prm = oracle_cycle_params(params)
    assert prm.kcycle_threshold == threshold and len(hier) >= 3
    r = W.random_complex(hier[0]["A"].shape[0], 16)
    z = op.vcycle(_cvec(r)).cpu().numpy()
    ref = mg.cycle(hier, r, prm)
    assert rel(z, ref) <= 1e-10, rel(z, ref)
    q = adr.point_source_rhs(adr.Grid(P.n, P.h), P.src)
    a, _ = op.solve(tol=0.0, maxit=6, raise_on_fail=False)
    x, _, _, _ = krylov.fgmres(oracle_matrix(name, "2up"), q, lambda v: mg.cycle(hier, v, prm), tol=0.0, restart=20,
                               maxit=6, reorth_eta=params.reorth_eta)
    assert rel(a.cpu().numpy(), x) <= 1e-10, rel(a.cpu().numpy(), x)


@pytest.mark.parametrize("name,restart,eta", [("marine2d_65", 8, 0.1), ("layered3d_17", 8, 0.1),
                                              ("corner3d_9x11x13", 4, 0.0), ("const3d_49x49x25", 8, 0.1),
                                              ("marine2d_65", 3, 2.0), ("layered3d_17", 5, 0.0)])
def test_double_float_outer_iteration(adrlib, cuda, name, restart, eta):
    """With a float32 cycle the outer iteration runs in double-float
    arithmetic on the float32 pipe (params.outer_df): A z_j, the selective
    Gram-Schmidt passes (never, selectively and always re-orthogonalised),
    the normalisation and x += Z y over several restarts.  Each operation
    differs from float64 at rounding level (2^-46 against 2^-53); the float32
    cycle turns such differences into float32-level ones now and then (an
    input within rounding of a float32 tie rounds the other way).  Within the
    first restart cycle that is rare and the iterates agree closely; each
    restart takes v_0 from the explicit residual, whose relative difference
    grows as the residual falls, so after several restarts iterates agree to
    the float32 cycle's precision only (measured 1.3e-6 after four restarts
    of FGMRES(3) on the 65^2 marine case); a wrong term would show at O(1).
    The precision check is the solve: to 1e-10 (where float32 arithmetic in
    the Krylov passes would stall near 1e-7) it reaches its explicit float64
    residual in the iterations of the float64 path (within one), and the two
    solutions agree to the solve's accuracy."""
    P, _, op_df = make_operator(name, precision="f32", levels=3, outer_df=1, restart=restart, reorth_eta=eta)
    _, _, op_64 = make_operator(name, precision="f32", levels=3, outer_df=0, restart=restart, reorth_eta=eta)
    for its, bound in ((restart, 1e-7), (12, 1e-5)):
        a1, _ = op_df.solve(tol=0.0, maxit=its, raise_on_fail=False)
        a0, _ = op_64.solve(tol=0.0, maxit=its, raise_on_fail=False)
        d = rel(a1.cpu().numpy(), a0.cpu().numpy())
        print(f"{name} FGMRES({restart}) eta {eta}: {its} iterations, iterates differ by {d:.2e}")
        assert d <= bound, (its, d)
    b1, i1 = op_df.solve(tol=1e-10, maxit=1000)
    b0, i0 = op_64.solve(tol=1e-10, maxit=1000)
    assert i1["rel_residual"] <= 1e-10 and abs(i1["iterations"] - i0["iterations"]) <= 1, (i1, i0)
    assert rel(b1.cpu().numpy(), b0.cpu().numpy()) <= 1e-8


@pytest.mark.parametrize("name", ["const2d_33", "marine2d_65", "layered3d_17"])
def test_cycle_f32(adrlib, cuda, name):
    """One float32 cycle against the oracle's float64 cycle.  Measured on
    GB300 (printed with -s): 3.0e-7 (const2d_33), 1.5e-6 (marine2d_65),
    2.5e-7 (layered3d_17), float32 rounding (6e-8) grown through the cycle's
    minimal-residual weights and coarse solves, which divide by inner
    products of near-cancelling Laplacian and reaction terms.  The bound 2e-5
    leaves a margin of about 13 over the largest; a wrong term or index shows
    at O(1)."""
    P, params, op = make_operator(name, precision="f32")
    hier = mg.build_hierarchy(oracle_matrix(name, "prec"), P.n, params.levels)
    r = W.random_complex(hier[0]["A"].shape[0], 12)
    z = op.vcycle(_cvec(r, torch.complex64)).cpu().numpy()
    ref = mg.cycle(hier, r, oracle_cycle_params(params))
    print(f"float32 cycle against the float64 oracle, {name}: {rel(z, ref):.2e}")
    assert rel(z, ref) <= 2e-5, rel(z, ref)


@pytest.mark.parametrize("name", ["const2d_33", "marine2d_65", "layered3d_17", "corner3d_9x11x13"])
@pytest.mark.parametrize("k,m", [(7, 20), (9, 4)])
@pytest.mark.parametrize("eta", [0.1, 2.0, 0.0])
def test_fgmres_iterates(adrlib, cuda, name, k, m, eta):
    """Same algorithm, fixed iteration count: iterate-for-iterate parity (selective,
    always and never re-orthogonalised Gram-Schmidt)."""
    P, params, op = make_operator(name, precision="f64", restart=m, reorth_eta=eta)
    A = oracle_matrix(name, "2up")
    hier = mg.build_hierarchy(oracle_matrix(name, "prec"), P.n, params.levels)
    prm = oracle_cycle_params(params)
    q = adr.point_source_rhs(adr.Grid(P.n, P.h), P.src)
    x_ref, its, res, _ = krylov.fgmres(A, q, lambda v: mg.cycle(hier, v, prm), tol=0.0, restart=m, maxit=k,
                                       reorth_eta=eta)
    a, info = op.solve(tol=0.0, maxit=k, raise_on_fail=False)
    assert info["iterations"] == its == k
    assert rel(a.cpu().numpy(), x_ref) <= 1e-10
    assert abs(info["rel_residual"] - res) <= 1e-8 * max(res, 1e-300) + 1e-14


@pytest.mark.parametrize("name", ["const2d_33", "ragged2d_37x21", "marine2d_65", "const3d_17x13x9", "layered3d_17"])
def test_solve_f64_to_direct(adrlib, cuda, name):
    P, params, op = make_operator(name, precision="f64")
    A = oracle_matrix(name, "2up")
    q = adr.point_source_rhs(adr.Grid(P.n, P.h), P.src)
    xe = spla.spsolve(A.tocsc(), q)
    a, info = op.solve(tol=1e-12, maxit=400)
    assert info["rel_residual"] <= 1e-12
    assert rel(a.cpu().numpy(), xe) <= 1e-10


@pytest.mark.parametrize("name", ["const2d_33", "marine2d_65", "layered3d_17"])
def test_solve_mixed_precision(adrlib, cuda, name):
    """float32 cycle inside the float64 FGMRES: the float64 residual still reaches 1e-8."""
    P, params, op = make_operator(name, precision="f32")
    A = oracle_matrix(name, "2up")
    q = adr.point_source_rhs(adr.Grid(P.n, P.h), P.src)
    a, info = op.solve(tol=1e-8, maxit=400)
    a = a.cpu().numpy()
    true_res = np.linalg.norm(q - A @ a) / np.linalg.norm(q)
    assert true_res <= 1.0000001e-8
    assert abs(true_res - info["rel_residual"]) <= 1e-12
    xe = spla.spsolve(A.tocsc(), q)
    # solution error bounded by the residual times the conditioning of H_2up
    assert rel(a, xe) <= 1e-5


@pytest.mark.parametrize("name", ["const2d_33", "marine2d_65", "layered3d_17"])
def test_solve_mixed_precision_refined(adrlib, cuda, name):
    """float32 cycle, float64 FGMRES continued to a 1e-12 residual (the outer
    loop refines the float32 preconditioner's output): the solution matches
    the direct solve of the oracle's H_2up to 1e-8 relative L2."""
    P, params, op = make_operator(name, precision="f32")
    A = oracle_matrix(name, "2up")
    q = adr.point_source_rhs(adr.Grid(P.n, P.h), P.src)
    a, info = op.solve(tol=1e-12, maxit=800)
    a = a.cpu().numpy()
    assert info["rel_residual"] <= 1e-12
    xe = spla.spsolve(A.tocsc(), q)
    err = rel(a, xe)
    print(f"mixed-precision refined {name}: {info['iterations']} iterations, residual {info['rel_residual']:.2e}, "
          f"error {err:.2e}")
    assert err <= 1e-8


def test_point_source_and_reconstruct(adrlib, cuda):
    P, _, op = make_operator("marine2d_65")
    g = adr.Grid(P.n, P.h)
    q = op.point_source_rhs().cpu().numpy()
    assert np.array_equal(q, adr.point_source_rhs(g, P.src))
    a = W.random_complex(g.N, 3)
    u = op.reconstruct(_cvec(a)).cpu().numpy()
    ref = adr.reconstruct(g, P.src, P.omega, P.tau1, a)
    assert np.abs(u - ref).max() <= 1e-13 * np.abs(ref).max()


def test_host_pipeline_matches_device(adrlib, cuda):
    from paper_1712_06091_gb300 import adr as gpu
    P, params, op = make_operator("marine2d_65")
    a_dev, info_dev = op.solve(tol=1e-8, maxit=300)
    u_dev = op.reconstruct(a_dev).cpu().numpy()
    u, a, info = gpu.solve_host(P.n, P.h, P.src, P.omega, P.kappa, P.tau1, P.gamma, params=params, tol=1e-8,
                                maxit=300, want_amplitude=True)
    assert info["iterations"] == info_dev["iterations"]
    assert np.array_equal(a, a_dev.cpu().numpy())
    assert np.array_equal(u, u_dev)


def test_not_converged_and_zero_rhs(adrlib, cuda):
    from paper_1712_06091_gb300 import adr as gpu
    P, params, op = make_operator("const2d_33")
    a, info = op.solve(tol=1e-14, maxit=2, raise_on_fail=False)
    assert info["status"] == gpu.L.ADR_ERR_NOT_CONVERGED and info["iterations"] == 2
    with pytest.raises(gpu.ADRError):
        op.solve(tol=1e-14, maxit=2)
    z = torch.zeros(op.N, dtype=torch.complex128, device="cuda")
    a, info = op.solve(rhs=z, tol=1e-8)
    assert info["iterations"] == 0 and torch.count_nonzero(a) == 0


@pytest.mark.parametrize("name,levels", [("marine2d_65", 2), ("layered3d_17", 2), ("const2d_33", 3),
                                         ("corner3d_9x11x13", 2)])
@pytest.mark.parametrize("form", ["kernels", "cta", "cluster", "grid"])
def test_coarse_solver_forms(adrlib, cuda, name, levels, form):
    """Every form of the coarsest-grid GMRES (one launch per step, one block,
    one cluster, one cooperative grid with barriers) against the oracle; the
    2-level cases put 1000-4000 nodes on the coarsest grid, several blocks of
    the cooperative form."""
    P, params, op = make_operator(name, precision="f64", levels=levels, coarse_solver=form)
    hier = mg.build_hierarchy(oracle_matrix(name, "prec"), P.n, params.levels)
    r = W.random_complex(hier[0]["A"].shape[0], 13)
    z = op.vcycle(_cvec(r)).cpu().numpy()
    assert rel(z, mg.cycle(hier, r, oracle_cycle_params(params))) <= 1e-10
    a, info = op.solve(tol=1e-10, maxit=400)
    xe = spla.spsolve(oracle_matrix(name, "2up").tocsc(), adr.point_source_rhs(adr.Grid(P.n, P.h), P.src))
    assert info["rel_residual"] <= 1e-10 and rel(a.cpu().numpy(), xe) <= 1e-8


@pytest.mark.parametrize("name", ["marine2d_65", "layered3d_17", "ragged2d_37x21", "corner3d_9x11x13"])
@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_bulk_copy_relaxation_matches_plain_loads(adrlib, cuda, name, variant):
    """The relaxation apply that streams coefficient tiles with bulk copies
    does each node's products as the plain-load kernel; the block sums of the
    minimal-residual weight follow its grid (and variants 3 and 4 add a node's
    terms in two or four groups), so cycles agree to float32 rounding and
    whole solves to their tolerance."""
    P, params, op_tma = make_operator(name, precision="f32", tma=variant, levels=3)
    _, _, op_plain = make_operator(name, precision="f32", tma=0, levels=3)
    r = _cvec(W.random_complex(P.N, 14), torch.complex64)
    z1, z0 = op_tma.vcycle(r).cpu().numpy(), op_plain.vcycle(r).cpu().numpy()
    assert rel(z1, z0) <= 1e-5
    a1, i1 = op_tma.solve(tol=1e-8)
    a0, i0 = op_plain.solve(tol=1e-8)
    assert abs(i1["iterations"] - i0["iterations"]) <= 1 and i1["rel_residual"] <= 1e-8
    assert rel(a1.cpu().numpy(), a0.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("variant,blocks", [(1, 1), (1, 2), (2, 1), (3, 1), (3, 2), (4, 1), (4, 2)])
def test_multi_tile_relaxation_loops_against_oracle(adrlib, cuda, variant, blocks):
    """The steady state of the streamed relaxation (buffer reuse, mbarrier phase
    flips, refills after the proxy fence) and of the finest-grid apply's
    grid-stride loop, against the oracle's cycle: relax_blocks caps both grids,
    so each warp of the bulk-copy kernel walks several level-1 tiles and each
    thread of the finest-grid apply walks ~235 nodes.  The float32 cycle must
    match the oracle's float64 cycle as closely as with the default grid
    (measured errors are reported by the assertion), and the two grids agree to
    float32 rounding of the weight's block sums."""
    name = "const3d_49x49x25"
    P, params, op = make_operator(name, precision="f32", tma=variant, levels=3, relax_blocks=blocks)
    n1 = op.info()["levels"][1]["nodes"]
    warps = 16 if variant == 1 else 8
    assert (n1 + 31) // 32 >= 7 * warps * blocks          # 254 tiles: 7 to 32 per warp
    hier = mg.build_hierarchy(oracle_matrix(name, "prec"), P.n, params.levels)
    r = W.random_complex(P.N, 15)
    z = op.vcycle(_cvec(r, torch.complex64)).cpu().numpy()
    ref = mg.cycle(hier, r, oracle_cycle_params(params))
    _, _, op0 = make_operator(name, precision="f32", tma=variant, levels=3)
    z0 = op0.vcycle(_cvec(r, torch.complex64)).cpu().numpy()
    e, e0 = rel(z, ref), rel(z0, ref)
    assert e <= 2e-4 and e <= 2.0 * e0 + 1e-6, (e, e0)
    assert rel(z, z0) <= 1e-5, rel(z, z0)
    # a whole solve with the capped grids reaches the tolerance in the same count
    a1, i1 = op.solve(tol=1e-8)
    a0, i0 = op0.solve(tol=1e-8)
    assert i1["rel_residual"] <= 1e-8 and abs(i1["iterations"] - i0["iterations"]) <= 1


# ---------------------------------------------------------------------------
# Eq. shift: the cycle built on the shifted operator; with tau1 = 0 the
# standard Helmholtz matrix with the shifted-Laplacian preconditioner (Sec. 3).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["const2d_33", "marine2d_65", "layered3d_17", "marine2d_65:helmholtz",
                                  "corner3d_9x11x13:helmholtz"])
@pytest.mark.parametrize("shift", [0.2, 0.5])
def test_shifted_preconditioner_apply(adrlib, cuda, name, shift):
    P, _, op = make_operator(name, shift=shift)
    A = oracle_matrix(name, "prec", shift=shift)
    x = W.random_complex(A.shape[0], 17)
    y = op.apply(_cvec(x), "prec").cpu().numpy()
    ref = A @ x
    assert np.abs(y - ref).max() / np.abs(ref).max() <= 1e-12
    # the outer operator does not see the shift
    y2 = op.apply(_cvec(x), "2up").cpu().numpy()
    ref2 = oracle_matrix(name, "2up") @ x
    assert np.abs(y2 - ref2).max() / np.abs(ref2).max() <= 1e-12


@pytest.mark.parametrize("name", ["marine2d_65", "marine2d_65:helmholtz", "layered3d_17:helmholtz"])
def test_shifted_cycle_f64(adrlib, cuda, name):
    P, params, op = make_operator(name, precision="f64", shift=0.2)
    hier = mg.build_hierarchy(oracle_matrix(name, "prec", shift=0.2), P.n, params.levels)
    r = W.random_complex(hier[0]["A"].shape[0], 19)
    z = op.vcycle(_cvec(r)).cpu().numpy()
    ref = mg.cycle(hier, r, oracle_cycle_params(params))
    assert rel(z, ref) <= 1e-10


@pytest.mark.parametrize("name", ["marine2d_65:helmholtz", "layered3d_17:helmholtz"])
def test_shifted_laplacian_fgmres_iterates(adrlib, cuda, name):
    """Standard Helmholtz (tau1 = 0, so H_2up = H) with the shifted-Laplacian
    cycle: fixed-count FGMRES iterates against the oracle."""
    P, params, op = make_operator(name, precision="f64", shift=0.2, restart=5)
    A = oracle_matrix(name, "2up")
    g = adr.Grid(P.n, P.h)
    H = adr.assemble_helmholtz(g, P.omega, P.kappa, P.gamma)
    assert abs(A - H).max() <= 1e-12 * abs(H).max()
    hier = mg.build_hierarchy(oracle_matrix(name, "prec", shift=0.2), P.n, params.levels)
    q = adr.point_source_rhs(g, P.src)
    x_ref, its, res, _ = krylov.fgmres(A, q, lambda v: mg.cycle(hier, v, oracle_cycle_params(params)), tol=0.0,
                                       restart=5, maxit=8, reorth_eta=params.reorth_eta)
    a, info = op.solve(tol=0.0, maxit=8, raise_on_fail=False)
    assert info["iterations"] == its == 8
    assert rel(a.cpu().numpy(), x_ref) <= 1e-10


@pytest.mark.parametrize("name", ["marine2d_65:helmholtz", "const3d_17x13x9:helmholtz"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_shifted_laplacian_solves_helmholtz(adrlib, cuda, name, precision):
    """The shifted-Laplacian solve of the standard Helmholtz system reaches 1e-8
    and the direct solution of H u = q."""
    P, params, op = make_operator(name, precision=precision, shift=0.2)
    g = adr.Grid(P.n, P.h)
    H = adr.assemble_helmholtz(g, P.omega, P.kappa, P.gamma)
    q = adr.point_source_rhs(g, P.src)
    u, info = op.solve(tol=1e-8, maxit=600)
    u = u.cpu().numpy()
    assert np.linalg.norm(q - H @ u) / np.linalg.norm(q) <= 1.0000001e-8
    assert rel(u, spla.spsolve(H.tocsc(), q)) <= 1e-4
