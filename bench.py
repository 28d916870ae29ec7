#!/usr/bin/env python
"""ADR amplitude solves per second to 1e-8 relative residual.

One step = the whole hot path for one point source on the 3D layered model
(257 x 257 x 129 nodes, 25 m spacing, 10 points per wavelength at the lowest
velocity): fine coefficients + Galerkin hierarchy (setup), flexible GMRES with
the multigrid preconditioner from a zero guess to |q - H_2up a| <= 1e-8 |q|,
and the reconstruction u = a exp(-i w tau).  The medium, tau1 and gamma are
resident in HBM before the timed region (tau1 comes from the library's own
travel-time kernel, outside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own source (independent problems, no
collective on the data path: weak scaling).  `--impl reference` times the CPU
oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADR solves/s to 1e-8 rel. residual at 256^2x128 cells (257x257x129 nodes)"
UNIT = "solves/s"
WORKLOADS = {
    "layered3d_257x257x129": dict(n=(257, 257, 129)),
    "layered3d_129x129x65": dict(n=(129, 129, 65)),
    "layered3d_65x65x33": dict(n=(65, 65, 33)),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="layered3d_257x257x129", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=400)
    ap.add_argument("--restart", type=int, default=None)
    ap.add_argument("--levels", type=int, default=None)
    ap.add_argument("--cycle", default=None)
    ap.add_argument("--sweeps", default=None, help="comma-separated relaxations per level")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def rank_source(n, rank):
    """Source position of rank r: lateral offsets around the centre, two nodes deep."""
    c0, c1 = (n[0] - 1) // 2, (n[1] - 1) // 2
    off = [(0, 0), (16, 0), (0, 16), (-16, 0), (0, -16), (16, 16), (-16, -16), (16, -16)][rank % 8]
    return (c0 + off[0], c1 + off[1], min(2, n[2] - 1))


def build_params(args):
    from paper_1712_06091_gb300 import adr as gpu
    kw = {"precision": args.precision}
    if args.restart:
        kw["restart"] = args.restart
    if args.levels:
        kw["levels"] = args.levels
    if args.cycle:
        kw["cycle"] = args.cycle
    if args.sweeps:
        kw["sweeps"] = [int(v) for v in args.sweeps.split(",")]
    return gpu.default_params(**kw)


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
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (the cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
SAMPLE_N = (33, 33, 17)


def oracle_sample(params_dict, tol):
    """One oracle solve (setup + FGMRES + cycle + reconstruction) on the layered 3D
    model resampled to 33 x 33 x 17 nodes.  Returns (seconds, nodes, iterations)."""
    from oracle import adr as oadr
    from oracle import eikonal, krylov
    from oracle import multigrid as omg
    from paper_1712_06091_gb300 import workloads as W
    P = W.layered_3d(SAMPLE_N)
    g = oadr.Grid(P.n, P.h)
    tau1 = eikonal.factored_fast_marching(g, P.kappa, P.src, order=2)
    t0 = time.perf_counter()
    A = oadr.assemble_adr(g, P.src, P.omega, P.kappa, P.gamma, tau1, "2up")
    Ap = oadr.assemble_preconditioner(g, P.src, P.omega, P.kappa, P.gamma, tau1, params_dict["beta"])
    hier = omg.build_hierarchy(Ap, P.n, params_dict["levels"])
    prm = omg.CycleParams(cycle=params_dict["cycle"], relax=params_dict["relax"], pre=params_dict["pre_sweeps"],
                          post=params_dict["post_sweeps"], weights=params_dict["jacobi_weight"],
                          coarse_iterations=params_dict["coarse_iterations"],
                          kcycle_iterations=params_dict["kcycle_iterations"])
    q = oadr.point_source_rhs(g, P.src)
    a, its, res, _ = krylov.fgmres(A, q, lambda v: omg.cycle(hier, v, prm), tol=tol,
                                   restart=params_dict["restart"], maxit=400)
    oadr.reconstruct(g, P.src, P.omega, tau1, a)
    return time.perf_counter() - t0, g.N, its


def cpu_rate_to_metric(seconds, nodes, its, full_nodes, full_its):
    """Oracle unknowns*iterations per second scaled to solves/s of the full workload."""
    rate = nodes * its / seconds
    return rate / (full_nodes * full_its)


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
    n = WORKLOADS[args.workload]["n"]
    src = rank_source(n, rank)
    P = W.layered_3d(n, src=src)
    params = build_params(args)
    stream = torch.cuda.current_stream(dev)
    kappa = torch.from_numpy(P.kappa).to(dev)
    gamma = torch.from_numpy(P.gamma).to(dev)
    tau1, sweeps = gpu.traveltime(P.n, P.h, P.src, kappa)
    op = gpu.Operator(P.n, P.h, P.src, P.omega, kappa, tau1, gamma, params=params, device=dev)
    a = torch.empty(P.N, dtype=torch.complex128, device=dev)

    def step():
        op.update(P.src, P.omega, kappa, tau1, gamma)
        _, info = op.solve(tol=args.tol, maxit=args.maxit, out=a)
        u = op.reconstruct(a)
        return info, u

    for _ in range(args.warmup):
        info, _ = step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches0 = gpu.kernel_launches()
    infos = []
    with ClockSampler(local) as clocks:
        t_wall = time.perf_counter()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            info, u = step()
            infos.append(info)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        if world > 1:
            dist.barrier()
    launches = gpu.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    its = [i["iterations"] for i in infos]
    res = max(i["rel_residual"] for i in infos)
    assert res <= args.tol, f"solve did not reach the tolerance: {res}"
    solves = args.steps * world
    value = solves / (ms / 1e3)

    # dominant-kernel roofline: the float64 outer apply of H_2up, timed by events on the op's stream
    peak_hbm, peak_kind = measured_peaks()
    x = torch.randn(P.N, dtype=torch.complex128, device=dev)
    for _ in range(3):
        op.apply(x, "2up")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(stream)
    for _ in range(reps):
        op.apply(x, "2up")
    e1.record(stream)
    torch.cuda.synchronize()
    k_ms = e0.elapsed_time(e1) / reps
    bytes_per_node = 16 + 16 + 8 * (2 * 3 + 2)
    achieved = bytes_per_node * P.N / (k_ms / 1e3) / 1e9

    e2e = None
    if not args.no_e2e and rank == 0:
        kh, th, gh = P.kappa, tau1.cpu().numpy(), P.gamma
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 3))
        for _ in range(e2e_steps):
            u_host, res_h = gpu.solve_host(P.n, P.h, P.src, P.omega, kh, th, gh, params=params, tol=args.tol,
                                           maxit=args.maxit)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e = {"value": e2e_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 3 * 8 * P.N,
               "d2h_bytes_per_step": 16 * P.N}

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        from paper_1712_06091_gb300.adr import params_dict
        secs, nodes, its_s = oracle_sample(params_dict(params), args.tol)
        cpu = {"value": cpu_rate_to_metric(secs, nodes, its_s, P.N, float(np.mean(its))), "unit": UNIT, "cores": 1,
               "kind": "oracle",
               "sample": f"one oracle solve (setup+FGMRES+cycle+reconstruct, tol {args.tol:g}) of the same model "
                         f"family at {SAMPLE_N[0]}x{SAMPLE_N[1]}x{SAMPLE_N[2]} nodes: {nodes} nodes x {its_s} its in "
                         f"{secs:.1f} s, scaled by unknowns*iterations to {P.N} nodes x {np.mean(its):.1f} its"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 cycle + f64 Krylov" if args.precision == "f32" else "f64",
            "data": "synthetic (seeded layered-gradient model with Gaussian anomalies; tau1 from the library's "
                    "travel-time kernel)",
            "config": {"workload": args.workload, "nodes": P.N, "grid": list(P.n), "spacing_km": P.h[0],
                       "omega": P.omega, "source": list(src), "tol": args.tol,
                       "params": gpu.params_dict(params), "iterations": its, "max_rel_residual": res,
                       "l2": "inputs and working set (several GB) larger than L2", "wall_s": t_wall,
                       "traveltime_sweeps": sweeps},
            "roofline": {"kernel": "k_fine_apply<3,double> (outer H_2up apply)", "bound": "hbm",
                         "achieved": achieved, "peak": peak_hbm, "unit": "GB/s", "frac": achieved / peak_hbm,
                         "peak_kind": peak_kind, "traffic": None, "bytes_per_node": bytes_per_node,
                         "launch_ms": k_ms},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks.summary(),
        }
        print(json.dumps(out))
    op.close()
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    """The CPU oracle as the reference arm (rank 0 only)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1712_06091_gb300 import adr as gpu_params_only  # parameter defaults only (no device work)
    import numpy as np
    params = gpu_params_only.params_dict(build_params(args))
    n = WORKLOADS[args.workload]["n"]
    N = int(np.prod(n))
    full_its = 30.0   # scaling assumption stated in the line: iterations of the full-size solve
    for _ in range(args.warmup):
        oracle_sample(params, args.tol)
    secs, its = [], []
    for _ in range(args.steps):
        s, nodes, k = oracle_sample(params, args.tol)
        secs.append(s)
        its.append(k)
    value = cpu_rate_to_metric(sum(secs), nodes * len(secs) // len(secs), float(np.mean(its)), N, full_its) * len(secs) / len(secs)
    value = (nodes * float(np.mean(its)) / float(np.mean(secs))) / (N * full_its)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "sample": list(SAMPLE_N), "assumed_full_iterations": full_its},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"oracle solve at {SAMPLE_N} nodes per step, scaled by unknowns*iterations"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
