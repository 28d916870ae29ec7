"""Launch-shape autotuner and packed multi-problem solves.

A set of point-source problems is solved in batches of problems that share a
grid (BatchOperator: one launch per step for the whole batch).  Two choices
are made by measurement on the device, not by rule:

* the packing: how many problems go into one batched operator (more problems
  per launch fill the GPU on the coarse levels and amortise launches, at the
  price of memory);
* the grid of the fused relaxation applies (params.relax_blocks): fewer
  blocks striding over more nodes against more blocks meeting at the
  reduction's ticket.

Each candidate runs a few outer iterations of the real solve (same problems,
same cycle) and is scored by device time per problem-iteration.
"""
from __future__ import annotations

import torch

from . import _lib as L
from . import adr as gpu

PACKINGS = (8, 16, 32)
RELAX_BLOCKS = (152, 304, 608, 1216, 2432)


def _stack(problems, k, device):
    return torch.stack([torch.as_tensor(p[k], dtype=torch.float64, device=device).reshape(-1) for p in problems])


def _params(params, **kw):
    p = L.Params.from_buffer_copy(params) if params is not None else gpu.default_params()
    for key, val in kw.items():
        setattr(p, key, val)
    return p


def probe(n, h, problems, params, iterations=3, repeats=2, device="cuda"):
    """Device ms per problem-iteration of a batched operator over `problems`
    (list of (src, omega, kappa, tau1, gamma)), `iterations` outer steps."""
    op = gpu.BatchOperator(n, h, [p[0] for p in problems], [p[1] for p in problems], _stack(problems, 2, device),
                           _stack(problems, 3, device), _stack(problems, 4, device), params=params, device=device)
    try:
        stream = op.stream
        op.solve(tol=0.0, maxit=iterations, raise_on_fail=False)          # warm-up (graph capture)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(repeats):
            op.solve(tol=0.0, maxit=iterations, raise_on_fail=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / (repeats * iterations * len(problems))
    finally:
        op.close()


def tune(n, h, problems, params=None, packings=PACKINGS, relax_blocks=RELAX_BLOCKS, iterations=3, device="cuda"):
    """Best (packing, relax_blocks) for these problems and the measured table.

    The relaxation grid is tuned first at the largest packing that the
    problem count allows, then the packing with that grid.
    """
    packings = [b for b in packings if b <= len(problems)] or [len(problems)]
    table = []
    b0 = max(packings)
    best_rb, best_t = None, float("inf")
    for rb in relax_blocks:
        t = probe(n, h, problems[:b0], _params(params, relax_blocks=rb), iterations, device=device)
        table.append({"packing": b0, "relax_blocks": rb, "ms_per_problem_iteration": t})
        if t < best_t:
            best_rb, best_t = rb, t
    best_b = b0
    for b in packings:
        if b == b0:
            continue
        t = probe(n, h, problems[:b], _params(params, relax_blocks=best_rb), iterations, device=device)
        table.append({"packing": b, "relax_blocks": best_rb, "ms_per_problem_iteration": t})
        if t < best_t:
            best_b, best_t = b, t
    return {"packing": best_b, "relax_blocks": best_rb, "ms_per_problem_iteration": best_t, "table": table}


class PackedSolver:
    """Solves a list of problems on one grid in batches of `packing` problems,
    reusing one BatchOperator per batch size (adr_batch_update between batches)."""

    def __init__(self, n, h, packing, params=None, device="cuda"):
        self.n, self.h, self.packing = tuple(n), tuple(h), int(packing)
        self.params = params if params is not None else gpu.default_params()
        self.device = torch.device(device)
        self._ops = {}

    def _op(self, chunk):
        b = len(chunk)
        args = ([p[0] for p in chunk], [p[1] for p in chunk], _stack(chunk, 2, self.device),
                _stack(chunk, 3, self.device), _stack(chunk, 4, self.device))
        op = self._ops.get(b)
        if op is None:
            op = gpu.BatchOperator(self.n, self.h, *args, params=self.params, device=self.device)
            self._ops[b] = op
        else:
            op.update(*args)
        return op

    def solve(self, problems, tol=1e-8, maxit=500, reconstruct=True):
        """(list of wavefields u (or amplitudes a) per problem, list of info dicts)."""
        out, infos = [], []
        for s in range(0, len(problems), self.packing):
            chunk = problems[s:s + self.packing]
            op = self._op(chunk)
            a, inf = op.solve(tol=tol, maxit=maxit)
            v = op.reconstruct(a) if reconstruct else a
            out.extend(v.reshape(len(chunk), -1).unbind(0))
            infos.extend(inf)
        return out, infos

    def close(self):
        for op in self._ops.values():
            op.close()
        self._ops.clear()


# ---------------------------------------------------------------------------
# Problems on grids of several sizes (GridsBatchOperator): one operator covers
# `packing` problems of every grid, so each launch of a step runs problems of
# all sizes together.
# ---------------------------------------------------------------------------
def _mixed_chunk(groups, start, packing):
    """Problems start .. start + packing of every group, as (grids, problems)."""
    grids, probs = [], []
    for (n, h), problems in groups:
        for p in problems[start:start + packing]:
            grids.append((n, h))
            probs.append(p)
    return grids, probs


def _cat(problems, k, device):
    return torch.cat([torch.as_tensor(p[k], dtype=torch.float64, device=device).reshape(-1) for p in problems])


def probe_grids(groups, packing, params, iterations=3, repeats=2, device="cuda"):
    """Device ms per problem-iteration of one mixed-grid operator holding
    `packing` problems of every group ((n, h), problems)."""
    grids, probs = _mixed_chunk(groups, 0, packing)
    op = gpu.GridsBatchOperator(grids, [p[0] for p in probs], [p[1] for p in probs], _cat(probs, 2, device),
                                _cat(probs, 3, device), _cat(probs, 4, device), params=params, device=device)
    try:
        stream = op.stream
        op.solve(tol=0.0, maxit=iterations, raise_on_fail=False)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(repeats):
            op.solve(tol=0.0, maxit=iterations, raise_on_fail=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / (repeats * iterations * len(probs))
    finally:
        op.close()


def tune_grids(groups, params=None, packings=PACKINGS, relax_blocks=RELAX_BLOCKS, iterations=3, device="cuda"):
    """Best (packing, relax_blocks) for mixed-grid operators over `groups`
    ((n, h), problems) and the measured table; as tune(), the relaxation grid
    first at the largest packing, then the packing."""
    count = min(len(p) for _, p in groups)
    packings = [b for b in packings if b <= count] or [count]
    table = []
    b0 = max(packings)
    best_rb, best_t = None, float("inf")
    for rb in relax_blocks:
        t = probe_grids(groups, b0, _params(params, relax_blocks=rb), iterations, device=device)
        table.append({"packing": b0, "relax_blocks": rb, "ms_per_problem_iteration": t})
        if t < best_t:
            best_rb, best_t = rb, t
    best_b = b0
    for b in packings:
        if b == b0:
            continue
        t = probe_grids(groups, b, _params(params, relax_blocks=best_rb), iterations, device=device)
        table.append({"packing": b, "relax_blocks": best_rb, "ms_per_problem_iteration": t})
        if t < best_t:
            best_b, best_t = b, t
    return {"packing": best_b, "relax_blocks": best_rb, "ms_per_problem_iteration": best_t, "table": table}


class GridsPackedSolver:
    """Solves problems on several grids with mixed-grid operators of `packing`
    problems per grid, reusing one operator per chunk shape (adr_batch_update
    between chunks)."""

    def __init__(self, packing, params=None, device="cuda"):
        self.packing = int(packing)
        self.params = params if params is not None else gpu.default_params()
        self.device = torch.device(device)
        self._ops = {}

    def solve(self, groups, tol=1e-8, maxit=500, reconstruct=True):
        """(per group: list of wavefields (or amplitudes) per problem, per group: list of info dicts)."""
        count = max(len(p) for _, p in groups)
        outs = [[] for _ in groups]
        infos = [[] for _ in groups]
        for s in range(0, count, self.packing):
            grids, probs = _mixed_chunk(groups, s, self.packing)
            key = tuple(grids)
            args = ([p[0] for p in probs], [p[1] for p in probs], _cat(probs, 2, self.device),
                    _cat(probs, 3, self.device), _cat(probs, 4, self.device))
            op = self._ops.get(key)
            if op is None:
                op = gpu.GridsBatchOperator(grids, *args, params=self.params, device=self.device)
                self._ops[key] = op
            else:
                op.update(*args)
            a, inf = op.solve(tol=tol, maxit=maxit)
            v = op.split(op.reconstruct(a) if reconstruct else a)
            k = 0
            for gi, ((n, h), problems) in enumerate(groups):
                for _ in problems[s:s + self.packing]:
                    outs[gi].append(v[k])
                    infos[gi].append(inf[k])
                    k += 1
        return outs, infos

    def close(self):
        for op in self._ops.values():
            op.close()
        self._ops.clear()
