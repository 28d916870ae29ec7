#!/usr/bin/env python
"""ADR amplitude solves per second to 1e-8 relative residual.

One step = the whole hot path for one point source on the 3D layered model
(257 x 257 x 129 nodes, 25 m spacing, 10 points per wavelength at the lowest
velocity): fine coefficients + stored outer rows + Galerkin hierarchy (setup),
flexible GMRES with the multigrid preconditioner from a zero guess to
|q - H_2up a| <= 1e-8 |q|, and the reconstruction u = a exp(-i w tau).  The
medium, tau1 and gamma are resident in HBM before the timed region (tau1 comes
from the library's own travel-time kernel, outside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own source (independent problems, no
collective on the data path: weak scaling).  `--impl reference` times the CPU
oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

# The oracle leg runs single-threaded so that `cores` below is what it used.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADR solves/s to 1e-8 rel. residual at 256^2x128 cells (257x257x129 nodes)"
UNIT = "solves/s"
SL_METRIC = ("standard Helmholtz solves/s (shifted-Laplacian cycle) to 1e-8 rel. residual at 256^2x128 cells "
             "(257x257x129 nodes)")
CEN_METRIC = ("central ADR solves/s (two-stage, Alg. ADRlong) to 1e-8 rel. residual at 256^2x128 cells "
              "(257x257x129 nodes)")
METHODS = ("adr-upwind", "helmholtz-sl", "adr-central")


def metric_for(args):
    return {"helmholtz-sl": SL_METRIC, "adr-central": CEN_METRIC}.get(args.method, METRIC)
WORKLOADS = {
    "layered3d_257x257x129": (257, 257, 129),
    "layered3d_193x193x97": (193, 193, 97),
    "layered3d_129x129x65": (129, 129, 65),
    "layered3d_65x65x33": (65, 65, 33),
}
# Cycle used by the bench: the paper's K-cycle with one-step Jacobi-GMRES
# relaxation (l+1 sweeps on level l), on 3 levels instead of the paper's 5
# (measured fastest on this workload; iteration counts are about the same).
BENCH_LEVELS = 3
# Outer FGMRES restart: 8 was fastest on GB300 at 257x257x129 (458 ms against
# 505 ms for 20, the same 70 iterations; 5, the paper's, took 73 iterations).
BENCH_RESTART = 8
# Grid of the finest-level relaxation applies: one resident wave (four blocks of
# 256 threads per SM), walked by grid-stride loops.  Measured at 257x257x129:
# 161 us per apply and 404 ms per solve against 176 us and 410 ms with the
# library default of 2432 blocks.
RELAX_BLOCKS_PER_SM = 4


def bench_relax_blocks():
    import torch
    if not torch.cuda.is_available():   # the oracle arm: the value only shapes GPU launches
        return 0
    return RELAX_BLOCKS_PER_SM * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


# Shifted-Laplacian comparison (Sec. 3, alpha = 0.2 as in Sec. 4); 4 levels
# measured fastest for it on the 257x257x129 model (49 iterations, against 75
# with 3 levels and 47 with 5 at a higher cost per cycle).
SL_SHIFT = 0.2
SL_LEVELS = 4
# Two-stage central solve (Alg. ADRlong): stage 1 to 1e-2 or 5 iterations
# (Sec. 4.2), stage 2 with the shifted cycle on the rescaled system.
CEN_LEVELS = 4
CEN_TOL1 = 1e-2
CEN_MAXIT1 = 5
CEN_FULL_ITERATIONS = 60.0   # stage 1 + stage 2 iterations of the GPU solve at 257x257x129 (measured)
# The kernel whose roofline is reported, and its algorithmic bytes per node of
# level 1: the 81-point stencil stored as 27 complex box entries and 54
# imaginary parts (float32), z and r read, w written (complex float32).
ROOFLINE_KERNEL = ("k_stencil_tma<3,float,false,16,kHalves,kTmaMr> on level 1 (minimal-residual relaxation apply, "
                   "81-point Galerkin stencil streamed into shared memory by bulk copies, each warp's tile buffer "
                   "refilled in halves)")
ROOFLINE_BYTES_PER_NODE = 27 * 8 + 54 * 4 + 3 * 8
# The finest-grid relaxation apply: packed rows (14 floats) plus z, r read and w written (complex float32).
FINE_RELAX_BYTES_PER_NODE = 14 * 4 + 3 * 8
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_stencil_tma_mr_level1_traffic.txt")
TRAFFIC_SOURCES = ["paper_1712_06091_gb300/csrc/coarse_tma.cu", "paper_1712_06091_gb300/csrc/coarse_stencil.cuh",
                   "paper_1712_06091_gb300/csrc/reduce.cuh", "paper_1712_06091_gb300/csrc/adr_common.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="layered3d_257x257x129", choices=list(WORKLOADS) + ["batched3d_3x32", "gradient3d_129_16src"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=400)
    ap.add_argument("--levels", type=int, default=None,
                    help=f"grid levels (default {BENCH_LEVELS} for the ADR solve, {SL_LEVELS} for the shifted Laplacian)")
    ap.add_argument("--method", default="adr-upwind", choices=list(METHODS),
                    help="adr-upwind: H_2up a = q with the (1-beta) H_2up + beta H_1up cycle; helmholtz-sl: the "
                         "standard Helmholtz matrix (tau1 = 0) with the shifted-Laplacian cycle (Eq. shift); "
                         "adr-central: H_cen a = q by the two-stage solve (Alg. ADRlong)")
    ap.add_argument("--shift", type=float, default=SL_SHIFT)
    ap.add_argument("--no-comparison", action="store_true")
    ap.add_argument("--no-breakdown", action="store_true",
                    help="skip the per-class live timing after the timed steps (one extra step per class) and the "
                         "whole-cycle roofline derived from it")
    ap.add_argument("--restart", type=int, default=None)
    ap.add_argument("--coarse-solver", default=None, choices=["auto", "kernels", "cta", "cluster", "grid"],
                    help="form of the coarsest-grid GMRES (same arithmetic; default: the library's choice)")
    ap.add_argument("--tma", type=int, default=None, choices=[0, 1, 2, 3, 4],
                    help="stored-stencil applies: 1 bulk copies, 16 warps; 2 bulk copies, 8 warps with two buffers; "
                         "3 (library default) / 4 bulk copies, 16 warps, buffers refilled in halves / quarters; "
                         "0 plain loads")
    ap.add_argument("--outer-df", type=int, default=None, choices=[0, 1],
                    help="outer Krylov iteration with the float32 cycle: 1 double-float (library default), 0 float64")
    ap.add_argument("--cycle", default=None)
    ap.add_argument("--sweeps", default=None, help="comma-separated relaxations per level")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-form", default="mixed", choices=["mixed", "per-grid"],
                    help="batched workload: one operator over problems of all grids (mixed) or one per grid")
    ap.add_argument("--paper-table", action="store_true",
                    help="probe only: the paper's solver configuration on two models at two resolutions each")
    ap.add_argument("--fp-rates", action="store_true",
                    help="probe only: float64 / float32 GEMM throughput of this GPU (no solve)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-sample", default="x".join(str(v) for v in SAMPLE_N),
                    help="grid of the oracle's bounded sample (cpu_baseline and --impl reference), e.g. 33x33x17")
    args = ap.parse_args()
    args.oracle_sample = tuple(int(v) for v in args.oracle_sample.split("x"))
    return args


def dist_env():
    from paper_1712_06091_gb300 import shard
    return shard.env()


def rank_source(n, rank):
    """Source of rank r: offsets around the lateral centre, two nodes deep."""
    c0, c1 = (n[0] - 1) // 2, (n[1] - 1) // 2
    off = [(0, 0), (16, 0), (0, 16), (-16, 0), (0, -16), (16, 16), (-16, -16), (16, -16)][rank % 8]
    return (c0 + off[0], c1 + off[1], min(2, n[2] - 1))


def build_params(args, method=None):
    """Parameters of the method's operators: [params] or, for the two-stage
    central solve, [stage 1, stage 2]."""
    from paper_1712_06091_gb300 import adr as gpu
    method = method or args.method
    levels = {"helmholtz-sl": SL_LEVELS, "adr-central": CEN_LEVELS}.get(method, BENCH_LEVELS)
    kw = {"precision": args.precision, "levels": args.levels or levels, "restart": args.restart or BENCH_RESTART,
          "relax_blocks": bench_relax_blocks()}
    if args.cycle:
        kw["cycle"] = args.cycle
    if args.coarse_solver:
        kw["coarse_solver"] = args.coarse_solver
    if args.tma is not None:
        kw["tma"] = args.tma
    if args.outer_df is not None:
        kw["outer_df"] = args.outer_df
    if args.sweeps:
        kw["sweeps"] = [int(v) for v in args.sweeps.split(",")]
    if method == "helmholtz-sl":
        return [gpu.default_params(shift=args.shift, **kw)]
    if method == "adr-central":
        return list(gpu.central_two_stage_params(shift=args.shift, **kw))
    return [gpu.default_params(**kw)]


class MethodSolver:
    """One step of a method on the bench medium and source: set up the
    operator(s) (coefficients and hierarchy), solve from zero to the
    tolerance, reconstruct u."""

    def __init__(self, method, P, kappa, tau1, gamma, args, dev):
        import torch
        from paper_1712_06091_gb300 import adr as gpu
        self.gpu, self.method, self.P, self.args = gpu, method, P, args
        self.kappa, self.gamma = kappa, gamma
        self.tau1 = torch.zeros_like(tau1) if method == "helmholtz-sl" else tau1   # tau = 0: u = a
        self.params = build_params(args, method)
        self.ops = [gpu.Operator(P.n, P.h, P.src, P.omega, kappa, self.tau1, gamma, params=p, device=dev)
                    for p in self.params]
        self.op = self.ops[-1]

    def step(self, out, marks=None):
        """One step; marks: optional [event, event] recorded after the setup and after the whole step (the
        caller records the start), on the operator's stream."""
        for op in self.ops:
            op.update(self.P.src, self.P.omega, self.kappa, self.tau1, self.gamma)
        if marks:
            marks[0].record(self.op.stream)
        if len(self.ops) == 1:
            _, info = self.op.solve(tol=self.args.tol, maxit=self.args.maxit, out=out)
        else:
            _, i1, i2 = self.gpu.solve_two_stage(self.ops[0], self.ops[1], tol1=CEN_TOL1, maxit1=CEN_MAXIT1,
                                                 tol=self.args.tol, maxit=self.args.maxit, out=out)
            info = dict(i2[0])
            info["stage1_iterations"] = i1[0]["iterations"]
            info["stage2_iterations"] = i2[0]["iterations"]
            info["iterations"] = i1[0]["iterations"] + i2[0]["iterations"]
        u = self.op.reconstruct(out)
        if marks:
            marks[1].record(self.op.stream)
        return info, u

    def close(self):
        for op in self.ops:
            op.close()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while active."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = [[p.strip() for p in line.split(",")] for line in open(self.path)]
        rows = [r for r in rows if len(r) >= 9]
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = sorted(v for v in (num(r[1]) for r in rows) if v is not None)
        mx = max((v for v in (num(r[2]) for r in rows) if v is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def nvtx_push(name):
    """Marks the timed region for `ncu --nvtx --nvtx-include timed/` (no-op without NVTX)."""
    import torch
    try:
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    import torch
    try:
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic_per_node():
    """DRAM bytes per level-1 node from the committed ncu summary, if the kernel is unchanged since."""
    if not os.path.exists(TRAFFIC_FILE):
        return None, "no ncu summary"
    d = {}
    with open(TRAFFIC_FILE) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                key, val = line.split(":", 1)
                d[key.strip()] = val.strip()
    if d.get("source_hash") != kernel_source_hash():
        return None, "kernel changed since the ncu capture"
    return float(d["dram_bytes_per_node"]), d.get("capture", "")


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (the cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
SAMPLE_N = (49, 49, 25)


def oracle_params(args, method=None):
    """The cycle and Krylov settings of the bench, as a plain dict for the
    oracle: the paper's K-cycle (Alg. Kcycle, FGMRES(2) inner steps), one
    Jacobi-GMRES step per relaxation with l+1 sweeps on level l (Sec. 4.2),
    10 coarsest GMRES steps, beta = 0.25 (Eq. precADRup), the bench's restart
    and level count.  The reference arm builds its oracle from this alone."""
    method = method or args.method
    levels = {"helmholtz-sl": SL_LEVELS, "adr-central": CEN_LEVELS}.get(method, BENCH_LEVELS)
    sweeps = [int(v) for v in args.sweeps.split(",")] if args.sweeps else [l + 2 for l in range(8)]
    sweeps = (sweeps + [sweeps[-1]] * 8)[:8]
    return {"levels": args.levels or levels, "beta": 0.25, "cycle": args.cycle or "K", "relax": "mr",
            "pre_sweeps": sweeps, "post_sweeps": list(sweeps), "jacobi_weight": [0.5] * 8,
            "coarse_iterations": 10, "kcycle_iterations": 2, "restart": args.restart or BENCH_RESTART,
            "reorth_eta": 0.1, "shift": args.shift if method in ("helmholtz-sl", "adr-central") else 0.0}


def oracle_sample(pd, tol, method="adr-upwind", n=None):
    """One oracle solve (setup + FGMRES + cycle + reconstruction) of the layered 3D model
    resampled to n nodes (default SAMPLE_N; helmholtz-sl: tau1 = 0 and the shifted cycle).
    Returns (seconds, nodes, iterations)."""
    import numpy as np
    from oracle import adr as oadr
    from oracle import eikonal, krylov
    from oracle import multigrid as omg
    from paper_1712_06091_gb300 import workloads as W
    P = W.layered_3d(tuple(n or SAMPLE_N))
    g = oadr.Grid(P.n, P.h)
    sl = method == "helmholtz-sl"
    tau1 = np.zeros(g.N) if sl else eikonal.factored_fast_marching(g, P.kappa, P.src, order=2)
    prm = omg.CycleParams(cycle=pd["cycle"], relax=pd["relax"], pre=pd["pre_sweeps"], post=pd["post_sweeps"],
                          weights=pd["jacobi_weight"], coarse_iterations=pd["coarse_iterations"],
                          kcycle_iterations=pd["kcycle_iterations"],
                          coarse_reorth_eta=pd["reorth_eta"] if pd["reorth_eta"] < 1.0 else None)
    t0 = time.perf_counter()
    if method == "adr-central":
        from oracle import twostage
        _, a, (its1, _), (its2, _) = twostage.two_stage_central(
            g, P.src, P.omega, P.kappa, P.gamma, tau1, prm, pd["levels"], alpha=pd["shift"], stage1_tol=CEN_TOL1,
            stage1_maxit=CEN_MAXIT1, tol=tol, restart=pd["restart"], maxit=400, reorth_eta=pd["reorth_eta"])
        oadr.reconstruct(g, P.src, P.omega, tau1, a)
        return time.perf_counter() - t0, g.N, its1 + its2
    A = oadr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, tau1, "2up")
    Ap = oadr.assemble_preconditioner(g, P.src, P.omega, P.kappa, P.gamma, tau1, pd["beta"], shift=pd.get("shift", 0.0))
    hier = omg.build_hierarchy(Ap, P.n, pd["levels"])
    q = oadr.point_source_rhs(g, P.src)
    a, its, res, _ = krylov.fgmres(A, q, lambda v: omg.cycle(hier, v, prm), tol=tol, restart=pd["restart"], maxit=400,
                                   reorth_eta=pd["reorth_eta"])
    oadr.reconstruct(g, P.src, P.omega, tau1, a)
    return time.perf_counter() - t0, g.N, its


def scale_to_workload(seconds, nodes, its, full_nodes, full_its):
    """Oracle unknowns*iterations per second, scaled to solves/s of the full workload."""
    return (nodes * its / seconds) / (full_nodes * full_its)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1712_06091_gb300 import adr as gpu
    from paper_1712_06091_gb300 import workloads as W

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    n = WORKLOADS[args.workload]
    src = rank_source(n, rank)
    P = W.layered_3d(n, src=src)
    stream = torch.cuda.current_stream(dev)
    kappa = torch.from_numpy(P.kappa).to(dev)
    gamma = torch.from_numpy(P.gamma).to(dev)
    # tau1 by the second-order factored eikonal on the device (input preparation, outside the timed region;
    # its own time is reported)
    gpu.traveltime(P.n, P.h, P.src, kappa, order=2)
    torch.cuda.synchronize()
    t_eik = time.perf_counter()
    tau1, sweeps = gpu.traveltime(P.n, P.h, P.src, kappa, order=2)
    torch.cuda.synchronize()
    t_eik = time.perf_counter() - t_eik
    solver = MethodSolver(args.method, P, kappa, tau1, gamma, args, dev)
    params = solver.params[-1]
    op = solver.op
    levels = op.info()["levels"]
    a = torch.empty(P.N, dtype=torch.complex128, device=dev)

    def step():
        return solver.step(a)

    # CUDA events around every launch of the roofline kernel (captured into the
    # cycle's graph, so enable before the warm-up; re-enabling resets the totals).
    op.profile("level1_relax")
    for _ in range(args.warmup):
        step()
    op.profile("level1_relax")
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches0 = gpu.kernel_launches()
    infos = []
    # per step: start, end of setup, end of step (events on the same stream, inside the timed region)
    marks = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    with ClockSampler(local) as clocks:
        t_wall = time.perf_counter()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        nvtx_push("timed")
        ev0.record(stream)
        for k in range(args.steps):
            marks[k][0].record(stream)
            info, _ = solver.step(a, marks[k][1:])
            infos.append(info)
        ev1.record(stream)
        torch.cuda.synchronize()
        nvtx_pop()
        t_wall = time.perf_counter() - t_wall
        if world > 1:
            dist.barrier()
    launches = gpu.kernel_launches() - launches0
    setup_ms = sum(m[0].elapsed_time(m[1]) for m in marks) / args.steps
    solve_ms = sum(m[1].elapsed_time(m[2]) for m in marks) / args.steps
    k_count, k_ms = op.profile_read()
    op.profile("none")
    from paper_1712_06091_gb300 import shard
    ms = shard.max_over_ranks(ev0.elapsed_time(ev1), device=dev)
    its = [i["iterations"] for i in infos]
    res = max(i["rel_residual"] for i in infos)
    assert res <= args.tol, f"solve did not reach the tolerance: {res}"
    value = args.steps * world / (ms / 1e3)

    peak, peak_kind = measured_peaks()
    n1 = levels[1]["nodes"] if len(levels) > 1 else 0
    per_launch_ms = k_ms / k_count if k_count else None
    achieved = ROOFLINE_BYTES_PER_NODE * n1 / (per_launch_ms / 1e3) / 1e9 if per_launch_ms else None
    tpn, traffic_note = measured_traffic_per_node()
    roofline = {"kernel": ROOFLINE_KERNEL, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "peak_kind": peak_kind,
                "traffic": tpn * n1 if tpn else None, "traffic_note": traffic_note,
                "algorithmic_bytes_per_launch": ROOFLINE_BYTES_PER_NODE * n1, "launches_timed": k_count,
                "avg_launch_ms": per_launch_ms}

    e2e = None
    if not args.no_e2e and rank == 0 and len(solver.ops) == 1:
        kh = torch.from_numpy(P.kappa).pin_memory().numpy()
        th = solver.tau1.cpu().pin_memory().numpy()
        gh = torch.from_numpy(P.gamma).pin_memory().numpy()
        uh = torch.empty(P.N, dtype=torch.complex128).pin_memory().numpy()
        torch.cuda.synchronize()
        e2e_steps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            _, res_h = gpu.solve_host(P.n, P.h, P.src, P.omega, kh, th, gh, params=params, tol=args.tol,
                                           maxit=args.maxit, out=uh)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        assert res_h["rel_residual"] <= args.tol, f"host-buffer solve did not reach the tolerance: {res_h}"
        e2e = {"value": e2e_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 3 * 8 * P.N,
               "d2h_bytes_per_step": 16 * P.N, "steps": e2e_steps,
               "note": "adr_solve_host: pinned host kappa/tau1/gamma in, host u out; operator built inside each call"}

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        secs, runs = 0.0, 0
        while secs < 10.0:      # at least ~10 s of oracle work
            s1, nodes, its_s = oracle_sample(oracle_params(args), args.tol, args.method, args.oracle_sample)
            secs, runs = secs + s1, runs + 1
        secs /= runs
        sn = "x".join(str(v) for v in args.oracle_sample)
        cpu = {"value": scale_to_workload(secs, nodes, its_s, P.N, float(np.mean(its))), "unit": UNIT, "cores": 1,
               "kind": "oracle",
               "extrapolated": f"by unknowns x iterations from {nodes} to {P.N} nodes",
               "sample": f"one oracle solve (setup + FGMRES + cycle + reconstruction, tol {args.tol:g}) of the same "
                         f"model family at {sn} nodes: {nodes} nodes x {its_s} iterations in {secs:.1f} s "
                         f"({nodes * its_s / secs:.3g} unknowns x iterations/s, one thread), scaled by "
                         f"unknowns*iterations to {P.N} nodes x {np.mean(its):.1f} iterations (mean of {runs} runs)"}

    breakdown = kernel_breakdown(solver, a) if not args.no_breakdown and rank == 0 else None

    cyc_roof = cycle_roofline(breakdown, levels, gpu.params_dict(params), peak, peak_kind)

    comparison = None
    if not args.no_comparison and rank == 0:
        comparison = [method_comparison(m, P, kappa, gamma, tau1, args, dev) for m in METHODS if m != args.method]
        if args.precision == "f32":     # the same method with the float64 cycle (the plain float64 solve)
            comparison.append(method_comparison(args.method, P, kappa, gamma, tau1, args, dev, precision="f64"))
            if outer_label(args) == "df64":   # the same FP32 cycle inside a float64 outer iteration
                comparison.append(method_comparison(args.method, P, kappa, gamma, tau1, args, dev, outer_df=0))

    if rank == 0:
        out = {
            "metric": metric_for(args), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_label(args),
            "data": "synthetic (seeded layered-gradient model with Gaussian anomalies; " +
                    ("tau1 = 0: the standard Helmholtz matrix)" if args.method == "helmholtz-sl" else
                     "tau1 from the library's second-order travel-time kernel)"),
            "method": args.method,
            "config": {"workload": args.workload, "method": args.method, "nodes": P.N, "grid": list(P.n), "spacing_km": P.h[0],
                       "omega": P.omega, "source": list(src), "tol": args.tol, "params": gpu.params_dict(params),
                       "levels": [lv["n"] for lv in levels], "iterations": its, "max_rel_residual": res,
                       "unknown_iterations_per_s": unknown_iterations_per_s(value, P.N, its),
                       "stage1_iterations": [i.get("stage1_iterations") for i in infos] if len(solver.ops) > 1 else None,
                       "l2": "no flush: inputs and working set (~9 GB) exceed L2", "wall_s": t_wall,
                       "traveltime_sweeps": sweeps, "traveltime_order": 2, "traveltime_ms": 1e3 * t_eik},
            "roofline": roofline,
            "cycle_roofline": cyc_roof,
            "setup_ms_per_step": setup_ms,
            "solve_ms_per_step": solve_ms,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks.summary(),
        }
        if comparison:
            out["comparison"] = comparison
        if breakdown:
            out["breakdown"] = breakdown
        print(json.dumps(out))
    solver.close()
    if world > 1:
        dist.destroy_process_group()


def unknown_iterations_per_s(solves_per_s, nodes, iterations):
    """Unknowns times outer iterations per second (the mean iteration count of the timed steps)."""
    return solves_per_s * nodes * (sum(iterations) / len(iterations))


def class_bandwidth(cls, us_per_launch, levels):
    """Algorithmic GB/s of a kernel class whose bytes per launch are fixed by its level's size (the two
    relaxation applies), else None."""
    if not us_per_launch:
        return None
    if cls == "level1_relax" and len(levels) > 1:
        bytes_per_launch = ROOFLINE_BYTES_PER_NODE * levels[1]["nodes"]
    elif cls == "fine_relax":
        bytes_per_launch = FINE_RELAX_BYTES_PER_NODE * levels[0]["nodes"]
    else:
        return None
    return bytes_per_launch / (us_per_launch * 1e-6) / 1e9


def cycle_bytes(levels, pd, dim=3):
    """Algorithmic bytes of one float32 preconditioner application (the K- or
    V-cycle with minimal-residual relaxation the bench runs), summed over the
    launches of the cycle in their order: every array a launch reads or
    writes counted once per launch (8 B per complex float32 entry, the packed
    finest-grid rows 4 (2 + 4 dim) B per node, the split Galerkin stencils
    (27 complex + 54 imaginary-only floats in 3D, 9 + 12 in 2D), no reuse
    between launches assumed).  The coarsest grid's bytes are counted the
    same way although its working set is L2-resident."""
    C = 8
    fine_rows = 4 * (2 + 4 * dim)
    stencil = (27 * 8 + 54 * 4) if dim == 3 else (9 * 8 + 12 * 4)
    N = [lv["nodes"] for lv in levels]
    L = len(N)

    def update(x_zero, has_next):       # x += alpha z ; r -= alpha w ; z_next = dinv r
        return (0 if x_zero else C) + C + 4 * C + (2 * C if has_next else 0)

    def relax(l, sweeps, x_zero):
        row = fine_rows if l == 0 else stencil
        b = 3 * C if x_zero else row + 5 * C                # D^{-1} b, or the residual with D^{-1}
        for s in range(sweeps):
            b += row + 3 * C + update(x_zero and s == 0, s + 1 < sweeps)
        return b * N[l]

    def coarse(l):
        k = pd["coarse_iterations"]
        n = N[l]
        b = C * n + 4 * C * n                                # |b|, V_0 and z = D^{-1} V_0
        for j in range(k):
            b += (stencil + 2 * C + (j + 1) * C) * n         # w = A z with the first pass's dots
            if pd.get("reorth_eta", 0.1) >= 1.0:             # the second pass (selective: not taken on
                b += (2 * C + 2 * (j + 1) * C) * n           # the bench's coarse operators, reading M2)
            if j + 1 < k:
                b += ((j + 1) * C + 5 * C) * n               # V_{j+1}, z
        return b + (k * C + 2 * C) * n                       # x = D^{-1} V y

    def cgs2(k, n):                                          # three passes over k basis vectors
        return (k * C + C + (2 * k * C + 2 * C) + (k * C + 2 * C)) * n

    def kcycle(l):
        k = pd["kcycle_iterations"]
        n = N[l]
        b = C * n + 2 * C * n                                # |b| and V_0
        for j in range(k):
            b += cycle(l)
            b += (stencil + 2 * C) * n + cgs2(j + 1, n)      # A z_j and its orthogonalisation
            if j + 1 < k:
                b += 2 * C * n
        return b + (k * C + C) * n                           # x = Z y

    def cycle(l):
        if l == L - 1:
            return coarse(l)
        b = relax(l, pd["pre_sweeps"][l], True)
        b += C * N[l] + C * N[l + 1]                         # restriction
        b += kcycle(l + 1) if pd["cycle"] == "K" and l + 1 < L - 1 else cycle(l + 1)
        b += C * N[l + 1] + 2 * C * N[l]                     # prolongation and correction
        return b + relax(l, pd["post_sweeps"][l], False)

    return cycle(0)


def kernel_breakdown(solver, a):
    """Live time of each instrumented kernel class inside a step: CUDA events
    around every launch of the class (event-record nodes in the captured
    cycle), one warm step to capture the instrumented graph, then one timed
    step per class.  Outside the bench's timed region."""
    import torch
    op = solver.op
    levels = op.info()["levels"]
    out = {}
    for cls in ("level1_relax", "fine_relax", "outer_apply", "coarsest", "cycle"):
        op.profile(cls)
        solver.step(a)
        op.profile(cls)
        solver.step(a)
        torch.cuda.synchronize()
        cnt, ms = op.profile_read()
        us = 1e3 * ms / cnt if cnt else None
        out[cls] = {"launches_per_step": cnt, "ms_per_step": ms, "us_per_launch": us,
                    "algorithmic_gbs": class_bandwidth(cls, us, levels)}
    op.profile("none")
    return out


def cycle_roofline(breakdown, levels, pd, peak, peak_kind):
    """The whole cycle against the HBM roofline: its algorithmic bytes (cycle_bytes)
    over the live duration of one cycle (CUDA events around each replay of the
    captured cycle inside a step)."""
    cyc = breakdown.get("cycle") if breakdown else None
    if not cyc or not cyc.get("us_per_launch") or pd["precision"] != "f32":
        return None
    b = cycle_bytes(levels, pd, len(levels[0]["n"]))
    gbs = b / (cyc["us_per_launch"] * 1e-6) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak, "peak_kind": peak_kind,
            "algorithmic_bytes_per_cycle": b, "cycles_per_step": cyc["launches_per_step"],
            "avg_cycle_ms": cyc["us_per_launch"] / 1e3,
            "note": "sum of the algorithmic bytes of every launch of one preconditioner application (model in "
                    "bench.cycle_bytes) over its live event time"}


def method_comparison(method, P, kappa, gamma, tau1, args, dev, precision=None, outer_df=None):
    """Another method (or the same one in another cycle or outer precision) on
    the same medium, source and tolerance (the paper's comparison of Sec. 4):
    one warm-up step, then one step (operator setup, solve, reconstruction)
    timed with CUDA events."""
    import copy
    import torch
    from paper_1712_06091_gb300 import adr as gpu
    if precision or outer_df is not None:
        args = copy.copy(args)
        args.precision = precision or args.precision
        args.outer_df = outer_df if outer_df is not None else args.outer_df
    solver = MethodSolver(method, P, kappa, tau1, gamma, args, dev)
    a = torch.empty(P.N, dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)
    solver.step(a)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    info, _ = solver.step(a)
    ev1.record(stream)
    torch.cuda.synchronize()
    out = {"method": method, "precision": args.precision, "outer": outer_label(args),
           "metric": {"helmholtz-sl": SL_METRIC, "adr-central": CEN_METRIC}.get(method, METRIC),
           "value": 1e3 / ev0.elapsed_time(ev1), "unit": UNIT, "ms_per_step": ev0.elapsed_time(ev1),
           "iterations": info["iterations"], "rel_residual": info["rel_residual"],
           "params": [gpu.params_dict(p) for p in solver.params]}
    if "stage1_iterations" in info:
        out["stage1_iterations"] = info["stage1_iterations"]
    solver.close()
    return out


def outer_label(args):
    """Arithmetic of the outer Krylov iteration: double-float with the float32
    cycle unless params.outer_df = 0 (float64 residual and solution either way)."""
    return "df64" if args.precision == "f32" and args.outer_df != 0 else "f64"


def dtype_label(args):
    if args.precision != "f32":
        return "f64"
    return "f32 cycle + " + ("df64 Krylov (f64 residual)" if outer_label(args) == "df64" else "f64 Krylov")


def run_reference(args):
    """The CPU oracle as the reference arm (rank 0 only).  Nothing here loads
    the CUDA library: the oracle's settings come from oracle_params."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    pd = oracle_params(args)
    N = int(np.prod(WORKLOADS[args.workload]))
    # iterations of the GPU solve at 257x257x129 with this cycle (bench config, measured)
    full_its = {"helmholtz-sl": 49.0, "adr-central": CEN_FULL_ITERATIONS}.get(args.method, 70.0)
    for _ in range(min(args.warmup, 1)):
        oracle_sample(pd, args.tol, args.method, args.oracle_sample)
    secs, its = [], []
    for _ in range(args.steps):
        s, nodes, k = oracle_sample(pd, args.tol, args.method, args.oracle_sample)
        secs.append(s)
        its.append(k)
    value = scale_to_workload(float(np.mean(secs)), nodes, float(np.mean(its)), N, full_its)
    sn = "x".join(str(v) for v in args.oracle_sample)
    sample = (f"oracle solve per step at {sn} nodes ({nodes} nodes x {np.mean(its):.0f} iterations in "
              f"{np.mean(secs):.1f} s, one thread), scaled by unknowns*iterations to {N} nodes x {full_its:.0f} "
              f"iterations")
    out = {"impl": "reference", "metric": metric_for(args), "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "sample": list(args.oracle_sample),
                      "assumed_full_iterations": full_its, "params": pd},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                            "extrapolated": f"by unknowns x iterations from {nodes} to {N} nodes"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# Batched multi-source workload: 32 surface sources on each of the 65^3, 97^3
# and 129^3 grids of the layered model (10 points per wavelength per grid,
# anisotropic spacing: 6.4 km laterally, 3.2 km deep), 96 solves per step.
# ---------------------------------------------------------------------------
BATCH_GRIDS = (65, 97, 129)
BATCH_SOURCES = 32
BATCH_METRIC = "ADR solves/s to 1e-8 rel. residual, 96 problems (32 sources x 65^3 / 97^3 / 129^3), batched"


def batch_problems(n, count, seed=3):
    """Model, and per source (src, omega, kappa, tau1, gamma) with tau1 from the device eikonal."""
    import numpy as np
    import torch
    from paper_1712_06091_gb300 import adr as gpu
    from paper_1712_06091_gb300 import workloads as W
    P = W.layered_3d((n, n, n))
    rng = np.random.default_rng(seed)
    lateral = rng.integers(2, n - 2, size=(count, 2))
    depth = rng.integers(1, 3, size=count)
    kappa = torch.from_numpy(P.kappa).cuda()
    out = []
    for (i0, i1), i2 in zip(lateral, depth):
        src = (int(i0), int(i1), int(i2))
        tau1, _ = gpu.traveltime(P.n, P.h, src, kappa, order=2)
        out.append((src, P.omega, kappa, tau1, torch.from_numpy(P.gamma).cuda()))
    return P, out


def run_batched(args):
    import torch
    import torch.distributed as dist
    from paper_1712_06091_gb300 import adr as gpu
    from paper_1712_06091_gb300 import autotune, shard
    rank, world, local = shard.env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    stream = torch.cuda.current_stream()
    groups = []
    for n in BATCH_GRIDS:
        # this rank's share of the grid's sources (independent problems: no exchange)
        mine = shard.partition(BATCH_SOURCES, rank, world)
        P, probs = batch_problems(n, BATCH_SOURCES)
        probs = [probs[i] for i in mine]
        params = gpu.default_params(precision="f32", levels=BENCH_LEVELS, restart=BENCH_RESTART)
        tuned = autotune.tune(P.n, P.h, probs, params=params) if args.batch_form == "per-grid" else None
        if tuned:
            params.relax_blocks = tuned["relax_blocks"]
        groups.append((P, probs, params, tuned))
    if args.batch_form == "mixed":
        # every launch of a step covers problems of all three grids (adr_batch_create_grids)
        mixed = [((P.n, P.h), probs) for P, probs, _, _ in groups]
        params = gpu.default_params(precision="f32", levels=BENCH_LEVELS, restart=BENCH_RESTART)
        mtuned = autotune.tune_grids(mixed, params=params)
        params.relax_blocks = mtuned["relax_blocks"]
        msolver = autotune.GridsPackedSolver(mtuned["packing"], params=params)
        solvers = [msolver]
    else:
        solvers = [autotune.PackedSolver(P.n, P.h, t["packing"], params=prm) for P, _, prm, t in groups]

    def step():
        if args.batch_form == "mixed":
            _, infos = msolver.solve(mixed, tol=args.tol, maxit=args.maxit)
            assert max(i["rel_residual"] for grp in infos for i in grp) <= args.tol
            return [[i["iterations"] for i in grp] for grp in infos]
        its = []
        for (P, probs, _, _), sol in zip(groups, solvers):
            _, infos = sol.solve(probs, tol=args.tol, maxit=args.maxit)
            assert max(i["rel_residual"] for i in infos) <= args.tol
            its.append([i["iterations"] for i in infos])
        return its

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = gpu.kernel_launches()
    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clocks:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            its = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    launches = gpu.kernel_launches() - launches0
    ms = shard.max_over_ranks(ev0.elapsed_time(ev1), device=dev)
    nprob = len(BATCH_GRIDS) * BATCH_SOURCES
    value = nprob * args.steps / (ms / 1e3)
    for s in solvers:
        s.close()

    # plain float64 reference: single-problem operators with the float64 cycle,
    # one source per grid, timed the same way and scaled to the 96 problems
    plain_ms = 0.0
    plain_its = []
    for P, probs, _, _ in groups:
        src, omega, kappa, tau1, gamma = probs[0]
        op = gpu.Operator(P.n, P.h, src, omega, kappa, tau1, gamma,
                          params=gpu.default_params(precision="f64", levels=BENCH_LEVELS, restart=BENCH_RESTART))
        op.solve(tol=args.tol, maxit=args.maxit)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(op.stream)
        _, info = op.solve(tol=args.tol, maxit=args.maxit)
        op.reconstruct(_)
        e1.record(op.stream)
        torch.cuda.synchronize()
        plain_ms += BATCH_SOURCES * e0.elapsed_time(e1)
        plain_its.append(info["iterations"])
        op.close()
    plain_value = nprob / (plain_ms / 1e3)
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    out = {
        "metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype_label(args), "data": "synthetic (layered model resampled per grid; tau1 from the library's "
                                                 "travel-time kernel)",
        "config": {"workload": "batched3d_3x32", "grids": list(BATCH_GRIDS), "sources_per_grid": BATCH_SOURCES,
                   "batch_form": args.batch_form,
                   "tuned": ([{"grids": "all", "packing_per_grid": mtuned["packing"],
                               "relax_blocks": mtuned["relax_blocks"], "table": mtuned["table"]}]
                             if args.batch_form == "mixed" else
                             [{"grid": P.n, "packing": t["packing"], "relax_blocks": t["relax_blocks"],
                               "table": t["table"]} for P, _, _, t in groups]),
                   "tol": args.tol,
                   "iterations_per_grid": [[min(i), max(i)] for i in its],
                   "l2": "no flush: batch working sets exceed L2"},
        "plain_f64": {"value": plain_value, "unit": UNIT, "iterations_per_grid": plain_its,
                      "note": "one single-problem solve per grid with the float64 cycle, scaled to 96 problems"},
        "speedup_vs_plain_f64": value / plain_value,
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    print(json.dumps(out))


# ---------------------------------------------------------------------------
# Adjoint gradient workload: misfit of 16 surface sources at 129 surface
# receivers on the 129^3 layered model, gradient with respect to the nodal
# slowness (travel time held fixed); data from a perturbed slowness.
# ---------------------------------------------------------------------------
GRAD_METRIC = "slowness-gradient evaluations/s (16 sources, 129^3, 129 receivers; forward + adjoint solves to 1e-8)"


def run_gradient(args):
    import numpy as np
    import torch
    from paper_1712_06091_gb300 import adr as gpu
    from paper_1712_06091_gb300 import workloads as W
    torch.cuda.set_device(0)
    n = 129
    P, probs = batch_problems(n, 16, seed=4)
    rec = torch.from_numpy((np.arange(n) + n * ((n - 1) // 2)).astype(np.int64)).cuda()   # surface line, mid i1
    kappa = probs[0][2]
    kappa_true = kappa * torch.from_numpy(1.0 + 0.02 * (W.smooth_random_field(P.n, seed=11) - 1.0)).cuda()
    params = gpu.default_params(precision="f32", levels=BENCH_LEVELS, restart=BENCH_RESTART)
    data = []
    for src, omega, _, tau1, gamma in probs:
        op = gpu.Operator(P.n, P.h, src, omega, kappa_true, tau1, gamma, params=params)
        a, _ = op.solve(tol=1e-10)
        data.append(op.reconstruct(a)[rec].clone())
        op.close()
    kw = dict(n=P.n, h=P.h, omega=P.omega, gamma=probs[0][4], sources=[p[0] for p in probs],
              tau1s=[p[3] for p in probs], receivers=rec, data=data, params=params, tol=args.tol, maxit=args.maxit)
    for _ in range(args.warmup):
        gpu.misfit_gradient(kappa=kappa, **kw)
    torch.cuda.synchronize()
    launches0 = gpu.kernel_launches()
    with ClockSampler(0) as clocks:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            J, grad = gpu.misfit_gradient(kappa=kappa, **kw)
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    out = {
        "metric": GRAD_METRIC, "value": args.steps / (ms / 1e3), "unit": "gradients/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 cycle + df64 Krylov (forward), f64 Krylov (adjoint)", "data": "synthetic (layered model; data from a 2% "
                                                                          "smooth slowness perturbation)",
        "config": {"workload": "gradient3d_129_16src", "grid": list(P.n), "sources": 16, "receivers": int(rec.numel()),
                   "tol": args.tol, "misfit": J, "grad_norm": float(grad.norm())},
        "gpu_launches": gpu.kernel_launches() - launches0, "clocks": clocks.summary(),
    }
    print(json.dumps(out))


PAPER_TABLE = (("marine2d", (257, 257)), ("marine2d", (513, 513)), ("layered3d", (129, 129, 65)),
               ("layered3d", (257, 257, 129)))


def run_paper_table(args):
    """The paper's own solver configuration (Sec. 4.2): flexible GMRES(5) to a
    1e-5 relative residual from zero, 5 levels of K-cycles (Alg. Kcycle, the
    0.1 coarse threshold, FGMRES(2) inner steps), Jacobi-GMRES relaxation with
    l+1 sweeps, 10 coarsest GMRES steps, beta = 0.25; the standard Helmholtz
    matrix with the shifted-Laplacian cycle (alpha = 0.2) beside it.  Runs the
    2D marine and 3D layered models at two resolutions each (10 points per
    wavelength, so the frequency doubles with the resolution) and prints the
    iteration counts and solve times (the trends of the paper's tables)."""
    import torch
    from paper_1712_06091_gb300 import adr as gpu
    from paper_1712_06091_gb300 import workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    rows = []
    for model, n in PAPER_TABLE:
        P = W.marine_2d(n) if model == "marine2d" else W.layered_3d(n)
        kappa = torch.from_numpy(P.kappa).to(dev)
        gamma = torch.from_numpy(P.gamma).to(dev)
        tau1, _ = gpu.traveltime(P.n, P.h, P.src, kappa, order=2)
        for method, tau, shift in (("adr-upwind", tau1, 0.0), ("helmholtz-sl", torch.zeros_like(tau1), 0.2)):
            prm = gpu.default_params(precision="f32", levels=5, restart=5, kcycle_threshold=0.1, shift=shift,
                                     relax_blocks=bench_relax_blocks())
            with gpu.Operator(P.n, P.h, P.src, P.omega, kappa, tau, gamma, params=prm, device=dev) as op:
                op.solve(tol=1e-5, maxit=1000)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(op.stream)
                a, info = op.solve(tol=1e-5, maxit=1000)
                e1.record(op.stream)
                torch.cuda.synchronize()
                rows.append({"model": model, "grid": list(P.n), "nodes": P.N, "method": method,
                             "ppw": P.meta.get("ppw"), "omega": P.omega, "iterations": info["iterations"],
                             "rel_residual": info["rel_residual"], "solve_ms": e0.elapsed_time(e1),
                             "levels": len(op.info()["levels"])})
    print(json.dumps({"probe": "paper_table", "config": "FGMRES(5), 5 levels, K-cycle (threshold 0.1), 1e-5, float32 "
                      "cycle", "rows": rows}))


def run_fp_rates(args):
    """Machine probe: float64 and float32 (TF32 off) throughput of square
    cuBLAS GEMMs through torch, best of several timed runs with CUDA events.
    The float64 figure bounds the library's float64 outer apply and
    Gram-Schmidt passes, which are arithmetic-bound on this GPU; the float32
    figure shows how far the float32 cycle is from its own ALU bound."""
    import torch
    torch.cuda.set_device(0)
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {"probe": "fp_rates", "unit": "TFLOP/s", "device": torch.cuda.get_device_name(0)}
    for name, dt, n in (("fp64", torch.float64, 8192), ("fp32", torch.float32, 8192)):
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        for _ in range(2):
            torch.matmul(a, b)
        best = None
        with ClockSampler(0) as clocks:
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
        out[name] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
        out[name + "_clocks"] = clocks.summary()
        del a, b
    print(json.dumps(out))


def main():
    args = parse()
    if args.fp_rates:
        run_fp_rates(args)
    elif args.paper_table:
        run_paper_table(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched3d_3x32":
        run_batched(args)
    elif args.workload == "gradient3d_129_16src":
        run_gradient(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
