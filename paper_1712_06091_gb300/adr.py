"""Python binding of libadr: same operations as include/adr.h, argument marshalling only.

Device memory and streams come from PyTorch; every computation runs in the
library's CUDA kernels.  Complex vectors are torch.complex128 (float64 path)
or torch.complex64 (float32 cycle), flat with N = prod(n) entries, axis 0
fastest.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L

ADRError = L.ADRError


def default_params(**overrides) -> L.Params:
    """adr_params_t with the library defaults, then `overrides` applied.

    Per-level lists (pre_sweeps, post_sweeps, jacobi_weight) may be given as
    Python sequences; cycle in {'V', 'K'}, relax in {'jacobi', 'mr'},
    precision in {'f64', 'f32'}.
    """
    p = L.Params()
    L.check(L.load().adr_params_default(ctypes.byref(p)))
    for key, val in overrides.items():
        if key == "cycle":
            p.cycle = L.CYCLES[val] if isinstance(val, str) else int(val)
        elif key == "relax":
            p.relax = L.RELAX[val] if isinstance(val, str) else int(val)
        elif key in ("scheme", "prec_scheme"):
            setattr(p, key, L.SCHEMES[val] if isinstance(val, str) else int(val))
        elif key == "coarse_solver":
            p.coarse_solver = L.COARSE_SOLVERS[val] if isinstance(val, str) else int(val)
        elif key in ("precision", "precond_precision"):
            p.precond_precision = {"f64": L.ADR_F64, "f32": L.ADR_F32}.get(val, val)
        elif key in ("pre_sweeps", "post_sweeps", "jacobi_weight"):
            arr = getattr(p, key)
            vals = list(val) if hasattr(val, "__len__") else [val] * L.MAX_LEVELS
            for k in range(L.MAX_LEVELS):
                arr[k] = vals[min(k, len(vals) - 1)]
        elif key == "sweeps":
            vals = list(val) if hasattr(val, "__len__") else [val] * L.MAX_LEVELS
            for k in range(L.MAX_LEVELS):
                p.pre_sweeps[k] = p.post_sweeps[k] = vals[min(k, len(vals) - 1)]
        else:
            setattr(p, key, val)
    return p


def params_dict(p: L.Params) -> dict:
    return {
        "levels": p.levels, "beta": p.beta, "cycle": "VK"[p.cycle], "relax": ["jacobi", "mr"][p.relax],
        "pre_sweeps": list(p.pre_sweeps), "post_sweeps": list(p.post_sweeps),
        "jacobi_weight": list(p.jacobi_weight), "coarse_iterations": p.coarse_iterations,
        "kcycle_iterations": p.kcycle_iterations, "restart": p.restart,
        "precision": ["f64", "f32"][p.precond_precision], "reorth_eta": p.reorth_eta,
        "relax_blocks": p.relax_blocks, "coarse_solver": p.coarse_solver, "tma": p.tma,
        "shift": p.shift, "scheme": _SCHEME_NAMES[p.scheme], "prec_scheme": _SCHEME_NAMES[p.prec_scheme],
        "rescale": p.rescale, "kcycle_threshold": p.kcycle_threshold, "outer_df": p.outer_df,
    }


_SCHEME_NAMES = {v: k for k, v in L.SCHEMES.items()}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _dev_real(x, N, device):
    t = torch.as_tensor(x, dtype=torch.float64, device=device).reshape(-1).contiguous()
    if t.numel() != N:
        raise ValueError(f"expected {N} values, got {t.numel()}")
    return t


class Operator:
    """H_2up and its multigrid hierarchy for one point source (adr_operator_create).

    tau_kind="factored" (default): `tau1` is the factor of tau = |x - x0| tau1;
    tau_kind="plain": `tau1` holds tau itself, differentiated by finite
    differences (adr_operator_create_tau; less accurate next to the source)."""

    def __init__(self, n, h, src, omega, kappa, tau1, gamma, params=None, device="cuda", stream=None,
                 tau_kind="factored"):
        self._lib = L.load()
        self.dim = len(n)
        self.n = tuple(int(v) for v in n)
        self.h = tuple(float(v) for v in h)
        self.src = tuple(int(v) for v in src)
        self.omega = float(omega)
        self.N = int(np.prod(self.n))
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.params = params if params is not None else default_params()
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        k = _dev_real(kappa, self.N, self.device)
        t = _dev_real(tau1, self.N, self.device)
        g = _dev_real(gamma, self.N, self.device)
        nn = (ctypes.c_int * 3)(*self.n, *([1] * (3 - self.dim)))
        hh = (ctypes.c_double * 3)(*self.h, *([1.0] * (3 - self.dim)))
        ss = (ctypes.c_int * 3)(*self.src, *([0] * (3 - self.dim)))
        handle = ctypes.c_void_p()
        if tau_kind not in ("factored", "plain"):
            raise ValueError("tau_kind must be 'factored' or 'plain'")
        create = self._lib.adr_operator_create_tau if tau_kind == "plain" else self._lib.adr_operator_create
        L.check(create(self.dim, nn, hh, ss, self.omega, _ptr(k), _ptr(t), _ptr(g), ctypes.byref(self.params),
                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle)))
        self._h = handle
        self.cycle_dtype = torch.complex128 if self.params.precond_precision == L.ADR_F64 else torch.complex64

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            L.check(self._lib.adr_operator_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def update(self, src, omega, kappa, tau1, gamma):
        """adr_operator_update: new source / frequency / medium, same grid and arena."""
        k = _dev_real(kappa, self.N, self.device)
        t = _dev_real(tau1, self.N, self.device)
        g = _dev_real(gamma, self.N, self.device)
        ss = (ctypes.c_int * 3)(*src, *([0] * (3 - self.dim)))
        L.check(self._lib.adr_operator_update(self._h, ss, float(omega), _ptr(k), _ptr(t), _ptr(g)))
        self.src = tuple(int(v) for v in src)
        self.omega = float(omega)

    def profile(self, kernel_class="none"):
        """adr_profile_kernel: time every launch of one kernel class with CUDA events."""
        L.check(self._lib.adr_profile_kernel(self._h, L.PROFILE_CLASSES[kernel_class]))

    def profile_read(self):
        """(launches timed, total milliseconds) since profile() was called."""
        n = ctypes.c_longlong(0)
        ms = ctypes.c_double(0.0)
        L.check(self._lib.adr_profile_read(self._h, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    # -- queries ----------------------------------------------------------
    def info(self) -> dict:
        i = L.OpInfo()
        L.check(self._lib.adr_operator_info(self._h, ctypes.byref(i)))
        levels = [{"n": tuple(i.level[l].n[: self.dim]), "nodes": i.level[l].nodes,
                   "stencil_points": i.level[l].stencil_points} for l in range(i.levels)]
        return {"dim": i.dim, "levels": levels, "arena_bytes": i.arena_bytes, "problems": i.problems}

    def coefficients(self) -> torch.Tensor:
        """(2*dim + 3, N) float64: d tau per axis, d^2 tau per axis, Re rho, Im rho, tau."""
        out = torch.empty((2 * self.dim + 3, self.N), dtype=torch.float64, device=self.device)
        L.check(self._lib.adr_coefficients(self._h, _ptr(out)))
        return out

    def level_stencil(self, level) -> torch.Tensor:
        info = self.info()["levels"][level]
        out = torch.empty((info["stencil_points"], info["nodes"]), dtype=self.cycle_dtype, device=self.device)
        L.check(self._lib.adr_level_stencil(self._h, int(level), _ptr(out)))
        return out

    # -- operations -------------------------------------------------------
    def _vec(self, x, dtype):
        if x.dtype != dtype or x.device != self.device or not x.is_contiguous() or x.numel() != self.N:
            raise ValueError(f"expected a contiguous {dtype} tensor of {self.N} entries on {self.device}")
        return x

    def apply(self, x, scheme="2up"):
        prec = L.ADR_F64 if x.dtype == torch.complex128 else L.ADR_F32
        x = self._vec(x.reshape(-1), x.dtype)
        y = torch.empty_like(x)
        L.check(self._lib.adr_apply(self._h, L.SCHEMES[scheme], prec, _ptr(x), _ptr(y)))
        return y

    def vcycle(self, r):
        r = self._vec(r.reshape(-1), self.cycle_dtype)
        z = torch.empty_like(r)
        L.check(self._lib.adr_vcycle(self._h, _ptr(r), _ptr(z)))
        return z

    def point_source_rhs(self):
        q = torch.empty(self.N, dtype=torch.complex128, device=self.device)
        L.check(self._lib.adr_point_source_rhs(self._h, _ptr(q)))
        return q

    def solve(self, rhs=None, x0=None, tol=1e-8, maxit=500, out=None, raise_on_fail=True):
        """(a, info dict).  rhs=None solves for the point source."""
        a = out if out is not None else torch.empty(self.N, dtype=torch.complex128, device=self.device)
        self._vec(a, torch.complex128)
        if x0 is not None:
            a.copy_(x0.reshape(-1))
        rp = ctypes.c_void_p(0) if rhs is None else _ptr(self._vec(rhs.reshape(-1), torch.complex128))
        info = L.SolveInfo()
        rc = self._lib.adr_solve(self._h, rp, _ptr(a), 1 if x0 is not None else 0, float(tol), int(maxit),
                                 ctypes.byref(info))
        allow = () if raise_on_fail else (L.ADR_ERR_NOT_CONVERGED,)
        L.check(rc, allow)
        return a, {"iterations": info.iterations, "restarts": info.restarts, "rel_residual": info.rel_residual,
                   "rel_estimate": info.rel_estimate, "status": info.status}

    # -- adjoint (operator created with params.adjoint = 1) ---------------
    def apply_adjoint(self, x):
        """adr_apply_adjoint: H_2up^H x (complex128)."""
        x = self._vec(x.reshape(-1), torch.complex128)
        y = torch.empty_like(x)
        L.check(self._lib.adr_apply_adjoint(self._h, _ptr(x), _ptr(y)))
        return y

    def vcycle_adjoint(self, r):
        """adr_vcycle_adjoint: one cycle on the conjugate-transposed hierarchy."""
        r = self._vec(r.reshape(-1), self.cycle_dtype)
        z = torch.empty_like(r)
        L.check(self._lib.adr_vcycle_adjoint(self._h, _ptr(r), _ptr(z)))
        return z

    def adjoint_solve(self, rhs, x0=None, tol=1e-8, maxit=500, out=None, raise_on_fail=True):
        """adr_adjoint_solve: (lambda, info) with H_2up^H lambda = rhs."""
        lam = out if out is not None else torch.empty(self.N, dtype=torch.complex128, device=self.device)
        self._vec(lam, torch.complex128)
        if x0 is not None:
            lam.copy_(x0.reshape(-1))
        rhs = self._vec(rhs.reshape(-1), torch.complex128)
        info = L.SolveInfo()
        rc = self._lib.adr_adjoint_solve(self._h, _ptr(rhs), _ptr(lam), 1 if x0 is not None else 0, float(tol),
                                         int(maxit), ctypes.byref(info))
        L.check(rc, () if raise_on_fail else (L.ADR_ERR_NOT_CONVERGED,))
        return lam, {"iterations": info.iterations, "restarts": info.restarts, "rel_residual": info.rel_residual,
                     "rel_estimate": info.rel_estimate, "status": info.status}

    def receivers(self, rec, d, u):
        """adr_receivers: (misfit 1/2 |u[rec] - d|^2, residuals, adjoint source M^H R^T res)."""
        rec = torch.as_tensor(rec, dtype=torch.int64, device=self.device).reshape(-1).contiguous()
        d = torch.as_tensor(d, dtype=torch.complex128, device=self.device).reshape(-1).contiguous()
        if d.numel() != rec.numel():
            raise ValueError("one datum per receiver")
        u = self._vec(u.reshape(-1), torch.complex128)
        res = torch.empty(rec.numel(), dtype=torch.complex128, device=self.device)
        rhs = torch.empty(self.N, dtype=torch.complex128, device=self.device)
        J = ctypes.c_double(0.0)
        L.check(self._lib.adr_receivers(self._h, int(rec.numel()), _ptr(rec), _ptr(d), _ptr(u), _ptr(res), _ptr(rhs),
                                        ctypes.byref(J)))
        return J.value, res, rhs

    def kappa_gradient(self, kappa, gamma, a, lam, grad):
        """adr_kappa_gradient: grad -= Re(conj(lam) dH/dkappa a) in place (float64, N)."""
        k = _dev_real(kappa, self.N, self.device)
        g = _dev_real(gamma, self.N, self.device)
        a = self._vec(a.reshape(-1), torch.complex128)
        lam = self._vec(lam.reshape(-1), torch.complex128)
        if grad.dtype != torch.float64 or grad.numel() != self.N or not grad.is_contiguous() or grad.device != self.device:
            raise ValueError("grad must be a contiguous float64 tensor of N entries on the operator's device")
        L.check(self._lib.adr_kappa_gradient(self._h, _ptr(k), _ptr(g), _ptr(a), _ptr(lam), _ptr(grad)))
        return grad

    def reconstruct(self, a):
        a = self._vec(a.reshape(-1), torch.complex128)
        u = torch.empty_like(a)
        L.check(self._lib.adr_reconstruct(self._h, _ptr(a), _ptr(u)))
        return u


def kernel_launches() -> int:
    """adr_kernel_launches: kernels launched by the library so far."""
    return int(L.load().adr_kernel_launches())


def traveltime(n, h, src, kappa, max_sweeps=None, device="cuda", stream=None, order=1):
    """adr_traveltime / adr_traveltime_order: device float64 tau1 for slowness
    `kappa` (factored eikonal, first- or second-order differences).  Returns
    (tau1, sweeps)."""
    lib = L.load()
    dim = len(n)
    N = int(np.prod(n))
    k = _dev_real(kappa, N, torch.device(device))
    tau1 = torch.empty(N, dtype=torch.float64, device=k.device)
    nn = (ctypes.c_int * 3)(*n, *([1] * (3 - dim)))
    hh = (ctypes.c_double * 3)(*h, *([1.0] * (3 - dim)))
    ss = (ctypes.c_int * 3)(*src, *([0] * (3 - dim)))
    st = stream if stream is not None else torch.cuda.current_stream(k.device)
    sweeps = ctypes.c_int(0)
    limit = max_sweeps if max_sweeps is not None else 8 * sum(n) + 64
    if order == 1:
        L.check(lib.adr_traveltime(dim, nn, hh, ss, _ptr(k), _ptr(tau1), int(limit), ctypes.c_void_p(st.cuda_stream),
                                   ctypes.byref(sweeps)))
    else:
        L.check(lib.adr_traveltime_order(dim, nn, hh, ss, _ptr(k), _ptr(tau1), int(order), int(limit),
                                         ctypes.c_void_p(st.cuda_stream), ctypes.byref(sweeps)))
    return tau1, sweeps.value


def solve_two_stage(stage1, stage2, rhs=None, tol1=1e-2, maxit1=5, tol=1e-8, maxit=500, out=None,
                    raise_on_fail=True):
    """adr_solve_two_stage (Alg. ADRlong): (a, [stage-1 infos], [stage-2 infos]).

    Stage 1 solves stage1's system from zero to tol1 or maxit1 iterations; its
    iterate starts stage 2's solve to tol.  Both are Operator / BatchOperator
    objects on the same grid, sources and frequencies."""
    B = getattr(stage1, "problems", 1)
    a = out if out is not None else torch.empty(stage2.N, dtype=torch.complex128, device=stage2.device)
    stage2._vec(a, torch.complex128)
    rp = ctypes.c_void_p(0) if rhs is None else _ptr(stage2._vec(rhs.reshape(-1), torch.complex128))
    info = (L.SolveInfo * (2 * B))()
    rc = stage2._lib.adr_solve_two_stage(stage1._h, stage2._h, rp, _ptr(a), float(tol1), int(maxit1), float(tol),
                                         int(maxit), info)
    L.check(rc, () if raise_on_fail else (L.ADR_ERR_NOT_CONVERGED,))
    d = [{"iterations": s.iterations, "restarts": s.restarts, "rel_residual": s.rel_residual,
          "rel_estimate": s.rel_estimate, "status": s.status} for s in info]
    return a, d[:B], d[B:]


def central_two_stage_params(**overrides):
    """Parameters of the two stages of Alg. ADRlong for the central ADR system:
    stage 1 = H_1up with its own cycle (beta = 1), stage 2 = H_cen with the
    shifted (alpha = 0.2, Sec. 4.2) cycle on the system rescaled as Helmholtz.
    `overrides` (cycle shape, precision, levels, restart, ...) apply to both;
    `shift` only to stage 2."""
    shift = overrides.pop("shift", 0.2)
    p1 = default_params(**overrides, scheme="1up", prec_scheme="prec", beta=1.0)
    p2 = default_params(**overrides, scheme="cen", prec_scheme="cen", shift=shift, rescale=1)
    return p1, p2


def solve_host(n, h, src, omega, kappa, tau1, gamma, params=None, tol=1e-8, maxit=500, stream=None,
               want_amplitude=False, out=None):
    """adr_solve_host: host numpy arrays in, host complex128 u (and a) out.

    `out` may be a preallocated (e.g. pinned) complex128 host array for u."""
    lib = L.load()
    dim = len(n)
    N = int(np.prod(n))
    k = np.ascontiguousarray(kappa, dtype=np.float64).reshape(-1)
    t = np.ascontiguousarray(tau1, dtype=np.float64).reshape(-1)
    g = np.ascontiguousarray(gamma, dtype=np.float64).reshape(-1)
    u = np.empty(N, dtype=np.complex128) if out is None else out
    if u.dtype != np.complex128 or u.size != N or not u.flags.c_contiguous:
        raise ValueError("out must be a contiguous complex128 array of N entries")
    a = np.empty(N, dtype=np.complex128) if want_amplitude else None
    p = params if params is not None else default_params()
    nn = (ctypes.c_int * 3)(*n, *([1] * (3 - dim)))
    hh = (ctypes.c_double * 3)(*h, *([1.0] * (3 - dim)))
    ss = (ctypes.c_int * 3)(*src, *([0] * (3 - dim)))
    st = ctypes.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    info = L.SolveInfo()
    rc = lib.adr_solve_host(dim, nn, hh, ss, float(omega), k.ctypes.data_as(ctypes.c_void_p),
                            t.ctypes.data_as(ctypes.c_void_p), g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(p),
                            float(tol), int(maxit), st, u.ctypes.data_as(ctypes.c_void_p),
                            a.ctypes.data_as(ctypes.c_void_p) if a is not None else ctypes.c_void_p(0),
                            ctypes.byref(info))
    L.check(rc)
    res = {"iterations": info.iterations, "restarts": info.restarts, "rel_residual": info.rel_residual,
           "status": info.status}
    return (u, a, res) if want_amplitude else (u, res)


def misfit_gradient(n, h, omega, kappa, gamma, sources, tau1s, receivers, data, params=None, tol=1e-10, maxit=500,
                    device="cuda", rank=None, world=None):
    """Receiver misfit J(kappa) = sum_s 1/2 |R u_s - d_s|^2 and dJ/dkappa (tau1 held fixed).

    Per source: adr_operator_update, adr_solve, adr_reconstruct, adr_receivers,
    adr_adjoint_solve, adr_kappa_gradient; one operator (a copy of params with
    adjoint = 1; the caller's params are not modified) is reused over the
    sources.  Under torch.distributed (or with rank / world given) every rank
    solves its `shard.partition` share of the sources and the misfit and
    gradient are summed over the ranks by one all-reduce, so every rank
    returns the full (J, grad).  Returns (J, grad) with grad a float64 tensor.
    """
    from . import shard
    device = torch.device(device)
    if device.type == "cuda" and device.index is None:
        device = torch.device("cuda", torch.cuda.current_device())
    p = L.Params.from_buffer_copy(params) if params is not None else default_params()
    p.adjoint = 1
    N = int(np.prod(n))
    k = _dev_real(kappa, N, device)
    g = _dev_real(gamma, N, device)
    grad = torch.zeros(N, dtype=torch.float64, device=device)
    a = torch.empty(N, dtype=torch.complex128, device=device)
    lam = torch.empty(N, dtype=torch.complex128, device=device)
    op = None

    def one_source(i):
        nonlocal op
        src, t1, d = sources[i], tau1s[i], data[i]
        if op is None:
            op = Operator(n, h, src, omega, k, t1, g, params=p, device=device)
        else:
            op.update(src, omega, k, t1, g)
        op.solve(tol=tol, maxit=maxit, out=a)
        u = op.reconstruct(a)
        Js, _, rhs = op.receivers(receivers, d, u)
        op.adjoint_solve(rhs, tol=tol, maxit=maxit, out=lam)
        op.kappa_gradient(k, g, a, lam, grad)    # accumulates into grad
        return Js, grad

    try:
        J, grad = shard.sharded_sum(len(sources), one_source, rank, world, out=grad)
    finally:
        if op is not None:
            op.close()
    return J, grad


class KappaMisfit(torch.autograd.Function):
    """J(kappa) as a differentiable scalar: forward runs the solves and the
    adjoint solves of misfit_gradient, backward scales the stored gradient.

        J = KappaMisfit.apply(kappa, problem)   # problem: dict of the other arguments
    """

    @staticmethod
    def forward(ctx, kappa, problem):
        J, grad = misfit_gradient(kappa=kappa.detach(), device=kappa.device, **problem)
        ctx.save_for_backward(grad.to(kappa.dtype))
        return torch.tensor(J, dtype=kappa.dtype, device=kappa.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return gJ * grad, None


class BatchOperator(Operator):
    """adr_batch_create: `problems` point-source problems on one grid, run together.

    Inputs and vectors are problem-major: kappa, tau1, gamma of shape
    (problems, N) (or flat problems * N); solve() returns a (problems * N)
    complex128 tensor and one info dict per problem.  `nodes` is N, `N` the
    total length of a batch vector.
    """

    def __init__(self, n, h, srcs, omegas, kappa, tau1, gamma, params=None, device="cuda", stream=None):
        self._lib = L.load()
        self.dim = len(n)
        self.n = tuple(int(v) for v in n)
        self.h = tuple(float(v) for v in h)
        self.problems = len(srcs)
        if len(omegas) != self.problems:
            raise ValueError("one frequency per source")
        self.srcs = [tuple(int(v) for v in s) for s in srcs]
        self.omegas = [float(w) for w in omegas]
        self.nodes = int(np.prod(self.n))
        self.N = self.nodes * self.problems
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.params = params if params is not None else default_params()
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        k = _dev_real(kappa, self.N, self.device)
        t = _dev_real(tau1, self.N, self.device)
        g = _dev_real(gamma, self.N, self.device)
        nn = (ctypes.c_int * 3)(*self.n, *([1] * (3 - self.dim)))
        hh = (ctypes.c_double * 3)(*self.h, *([1.0] * (3 - self.dim)))
        ss, ww = self._src_omega(self.srcs, self.omegas)
        handle = ctypes.c_void_p()
        L.check(self._lib.adr_batch_create(self.dim, nn, hh, self.problems, ss, ww, _ptr(k), _ptr(t), _ptr(g),
                                           ctypes.byref(self.params), ctypes.c_void_p(self.stream.cuda_stream),
                                           ctypes.byref(handle)))
        self._h = handle
        self.cycle_dtype = torch.complex128 if self.params.precond_precision == L.ADR_F64 else torch.complex64
        self.src = self.srcs[0]
        self.omega = self.omegas[0]

    def _src_omega(self, srcs, omegas):
        if len(srcs) != self.problems or len(omegas) != self.problems:
            raise ValueError(f"expected {self.problems} sources and frequencies")
        ss = (ctypes.c_int * (3 * self.problems))()
        for p, s in enumerate(srcs):
            for d in range(self.dim):
                ss[3 * p + d] = int(s[d])
        ww = (ctypes.c_double * self.problems)(*[float(w) for w in omegas])
        return ss, ww

    def update(self, srcs, omegas, kappa, tau1, gamma):
        """adr_batch_update: new sources / frequencies / media, same grid and arena."""
        k = _dev_real(kappa, self.N, self.device)
        t = _dev_real(tau1, self.N, self.device)
        g = _dev_real(gamma, self.N, self.device)
        ss, ww = self._src_omega(srcs, omegas)
        L.check(self._lib.adr_batch_update(self._h, ss, ww, _ptr(k), _ptr(t), _ptr(g)))
        self.srcs = [tuple(int(v) for v in s) for s in srcs]
        self.omegas = [float(w) for w in omegas]

    def coefficients(self) -> torch.Tensor:
        out = torch.empty((self.problems, 2 * self.dim + 3, self.nodes), dtype=torch.float64, device=self.device)
        L.check(self._lib.adr_coefficients(self._h, _ptr(out)))
        return out

    def level_stencil(self, level) -> torch.Tensor:
        info = self.info()["levels"][level]
        out = torch.empty((self.problems, info["stencil_points"], info["nodes"]), dtype=self.cycle_dtype,
                          device=self.device)
        L.check(self._lib.adr_level_stencil(self._h, int(level), _ptr(out)))
        return out

    def solve(self, rhs=None, x0=None, tol=1e-8, maxit=500, out=None, raise_on_fail=True):
        """(a, [info dict per problem]).  rhs=None solves for the point sources."""
        a = out if out is not None else torch.empty(self.N, dtype=torch.complex128, device=self.device)
        self._vec(a, torch.complex128)
        if x0 is not None:
            a.copy_(x0.reshape(-1))
        rp = ctypes.c_void_p(0) if rhs is None else _ptr(self._vec(rhs.reshape(-1), torch.complex128))
        infos = (L.SolveInfo * self.problems)()
        rc = self._lib.adr_solve(self._h, rp, _ptr(a), 1 if x0 is not None else 0, float(tol), int(maxit), infos)
        L.check(rc, () if raise_on_fail else (L.ADR_ERR_NOT_CONVERGED,))
        return a, [{"iterations": i.iterations, "restarts": i.restarts, "rel_residual": i.rel_residual,
                    "rel_estimate": i.rel_estimate, "status": i.status} for i in infos]


class GridsBatchOperator(BatchOperator):
    """adr_batch_create_grids: point-source problems with grids (and spacings)
    of their own, run together (each launch covers every problem).

    grids: one (n, h) pair per problem.  Inputs and vectors are the problems'
    node arrays concatenated in order (problem p's N_p entries after the
    earlier problems'); `offsets[p]` is where problem p starts and `N` the
    total length.  split(v) returns the per-problem views of such a vector.
    """

    def __init__(self, grids, srcs, omegas, kappa, tau1, gamma, params=None, device="cuda", stream=None):
        self._lib = L.load()
        if not grids:
            raise ValueError("at least one problem")
        self.dim = len(grids[0][0])
        self.grids = [(tuple(int(v) for v in n), tuple(float(v) for v in h)) for n, h in grids]
        if any(len(n) != self.dim or len(h) != self.dim for n, h in self.grids):
            raise ValueError("every grid needs dim node counts and spacings")
        self.problems = len(self.grids)
        if len(srcs) != self.problems or len(omegas) != self.problems:
            raise ValueError("one source and one frequency per grid")
        self.n, self.h = self.grids[0]
        self.srcs = [tuple(int(v) for v in s) for s in srcs]
        self.omegas = [float(w) for w in omegas]
        sizes = [int(np.prod(n)) for n, _ in self.grids]
        self.offsets = [int(v) for v in np.concatenate([[0], np.cumsum(sizes)[:-1]])]
        self.sizes = sizes
        self.nodes = max(sizes)
        self.N = int(sum(sizes))
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.params = params if params is not None else default_params()
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        k = _dev_real(kappa, self.N, self.device)
        t = _dev_real(tau1, self.N, self.device)
        g = _dev_real(gamma, self.N, self.device)
        nn = (ctypes.c_int * (3 * self.problems))()
        hh = (ctypes.c_double * (3 * self.problems))()
        for p, (n, h) in enumerate(self.grids):
            for d in range(3):
                nn[3 * p + d] = n[d] if d < self.dim else 1
                hh[3 * p + d] = h[d] if d < self.dim else 1.0
        ss, ww = self._src_omega(self.srcs, self.omegas)
        handle = ctypes.c_void_p()
        L.check(self._lib.adr_batch_create_grids(self.dim, self.problems, nn, hh, ss, ww, _ptr(k), _ptr(t), _ptr(g),
                                                 ctypes.byref(self.params), ctypes.c_void_p(self.stream.cuda_stream),
                                                 ctypes.byref(handle)))
        self._h = handle
        self.cycle_dtype = torch.complex128 if self.params.precond_precision == L.ADR_F64 else torch.complex64
        self.src = self.srcs[0]
        self.omega = self.omegas[0]

    def split(self, v):
        """Per-problem views of a concatenated batch vector."""
        v = v.reshape(-1)
        return [v[o:o + s] for o, s in zip(self.offsets, self.sizes)]

    def coefficients(self) -> torch.Tensor:
        """(2 dim + 3) N_p values per problem, concatenated (see adr_coefficients)."""
        out = torch.empty((2 * self.dim + 3) * self.N, dtype=torch.float64, device=self.device)
        L.check(self._lib.adr_coefficients(self._h, _ptr(out)))
        return out
