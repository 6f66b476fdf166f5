"""Autotuner of the batched solver: the column pass and its tile width per grid-size bucket, the
number of concurrent worker streams and the lockstep group size, each chosen by timing real solves of
the caller's own problems on the device (CUDA events), keeping the fastest."""
from __future__ import annotations

import collections

import torch

from . import binding as B


def _time(fn, reps=3):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def tune_tiles(geoms, solve_one, widths=(2, 4, 8), reps=2):
    """For each grid-size bucket, the tile width with the fastest solve of the bucket's first
    problem; `solve_one(k)` solves problem k.  Applies the choice to every geometry and returns
    {(nx, ny): width}."""
    buckets = collections.defaultdict(list)
    for k, g in enumerate(geoms):
        buckets[(g.grid.nx, g.grid.ny)].append(k)
    best = {}
    for key, ks in buckets.items():
        k0 = ks[0]
        times = {}
        for w in widths:
            B.iim_geometry_set_tiles(geoms[k0], w)
            times[w] = _time(lambda: solve_one(k0), reps)
        best[key] = min(times, key=times.get)
        for k in ks:
            B.iim_geometry_set_tiles(geoms[k], best[key])
    return best


def tune_tiles_batch(geoms, run_batch, widths=(4, 8), reps=2):
    """One tile width for all geometries, chosen by timing the whole batch `run_batch()` (the
    throughput mode: the best width for one solve alone need not be the best when many share
    the GPU).  Applies the choice and returns (width, {width: ms})."""
    times = {}
    for w in widths:
        for g in geoms:
            B.iim_geometry_set_tiles(g, w)
        run_batch()                     # the solve graphs are rebuilt for the new kernels
        times[w] = _time(run_batch, reps)
    best = min(times, key=times.get)
    for g in geoms:
        B.iim_geometry_set_tiles(g, best)
    return best, times


def tune_column_solver(geoms, run_batch, modes=(1, 0), reps=2, rebuild_precond=False):
    """One column pass for all geometries (iim_geometry_set_column_solver: 1 tridiagonal scans,
    0 column DSTs), chosen by timing the whole batch `run_batch()`: the passes differ in speed and
    in FP32 rounding, and the rounding can change how many refinements a solve takes.  With
    `rebuild_precond` each candidate also rebuilds the dense Schur preconditioner with its own
    column pass (the preconditioner's FP32 rounding matters too).  Applies the choice and returns
    (mode, {mode: ms})."""
    times = {}

    def apply(m):
        for g in geoms:
            B.iim_geometry_set_column_solver(g, m)
            if rebuild_precond:
                B.iim_build_preconditioner(g)

    for m in modes:
        apply(m)
        run_batch()
        times[m] = _time(run_batch, reps)
    best = min(times, key=times.get)
    apply(best)
    return best, times


def tune_streams(run_batch, candidates=(1, 2, 4, 8, 12, 16, 24)):
    """The number of worker streams for which `run_batch(n_streams)` is fastest."""
    times = {c: _time(lambda: run_batch(c), 1) for c in candidates}
    return min(times, key=times.get), times


def tune_lockstep(run_batch, candidates=(1, 2, 4, 8), reps=3):
    """The largest lockstep group (iim_set_lockstep; 1 = one whole-solve graph per problem) for
    which `run_batch()` is fastest.  Each candidate is run once untimed (its group graphs are
    captured then).  Applies the choice and returns (size, {size: ms})."""
    times = {}
    for c in candidates:
        B.iim_set_lockstep(c)
        run_batch()
        times[c] = _time(run_batch, reps)
    best = min(times, key=times.get)
    B.iim_set_lockstep(best)
    return best, times
