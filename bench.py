#!/usr/bin/env python3
"""Benchmark of the IIM Poisson hot path: solves/s on the single-cylinder workload at 1024^2
cells to a relative un-reduced residual of 1e-10 (chosen form: FP32 transforms inside FP64
iterative refinement), with the plain FP64 iteration timed beside it.

One step = one iim_poisson_solve (omega -> psi, u) through the C ABI with inputs resident in
HBM.  L2 is flushed (256 MiB write) before every timed step; the flush is outside the step's
CUDA events.  Under torchrun each rank runs independent solves on its own GPU (replicas, weak
scaling); rank 0 prints one JSON line.

--impl reference times the CPU oracle (Schur-form GMRES with scipy's DST-I, FP64) on the
host cores on the same workload, metric and unit.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IIM Poisson solves/s at 1024² to 1e-10 residual: chosen form vs plain FP64"
UNIT = "solves/s"
N_CELLS = 1024
RTOL = 1e-10
WORKLOAD = ("c1_cylinder_1024: [-2,2]^2, 1024x1024 cells (1023^2 unknowns), one cylinder R=0.5 at the origin, "
            "manufactured psi = sin(pi x/2) sin(pi y/2) + 0.1 log r, Dirichlet box and body data from psi, "
            "fixed-psibar body, solve to un-reduced FP64 relative residual 1e-10")
# DRAM traffic per launch of the dominant kernel from the committed ncu capture, valid for
# the kernel source hash below (null otherwise).
NCU_TRAFFIC = {}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("dst.cuh", "solve.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2109_13628_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_CELLS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--inner-rtol", type=float, default=0.0, help="mixed-mode Krylov tolerance (0: library default)")
    ap.add_argument("--restart", type=int, default=64)
    ap.add_argument("--sweep", action="store_true", help="print iterations/time for a grid of inner tolerances and exit")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
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
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def cpu_baseline(n, budget_s=20.0):
    """The oracle as it stands (Schur-form GMRES, scipy DST-I, FP64) on this host."""
    import numpy as np

    from oracle import poisson as op
    from paper_2109_13628_gb300 import inputs
    P = inputs.c1_cylinder(n)
    S = op.Setup(P)
    O = op.SchurOperators(S)
    done, t0 = 0, time.perf_counter()
    res = None
    while True:
        psi, pb, it, rel = op.solve_schur(S, psibar=np.zeros(1), tol=RTOL / 10, ops=O)
        done += 1
        el = time.perf_counter() - t0
        if el > budget_s or done >= 8:
            break
    res = op.residual(S, psi, pb)
    return {"value": done / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} oracle solves of the {n}^2 single-cylinder workload (GMRES {it} iterations, "
                      f"residual {res:.2e}), geometry setup excluded, {el:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    from oracle import poisson as op
    from paper_2109_13628_gb300 import inputs
    P = inputs.c1_cylinder(args.n)
    S = op.Setup(P)
    O = op.SchurOperators(S)
    for _ in range(args.warmup):
        op.solve_schur(S, psibar=np.zeros(1), tol=RTOL / 10, ops=O)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        psi, pb, it, rel = op.solve_schur(S, psibar=np.zeros(1), tol=RTOL / 10, ops=O)
    el = time.perf_counter() - t0
    v = args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step one full oracle solve ({it} GMRES iterations, FP64, scipy DST-I)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    import paper_2109_13628_gb300 as iim
    from paper_2109_13628_gb300 import inputs

    P = inputs.c1_cylinder(args.n)
    g = P.grid
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    grid = iim.make_grid(g.x0, g.x1, g.y0, g.y1, g.nx, g.ny)
    t_setup = time.perf_counter()
    geo = iim.iim_setup_geometry(grid, T(P.phi), P.regions, P.modes)
    t_setup = time.perf_counter() - t_setup
    cp = iim.iim_geometry_control_points(geo)
    psi_b_h = P.psi_b_fn(cp["x"].cpu().numpy(), cp["y"].cpu().numpy(), None)
    NXY = (g.nx - 1) * (g.ny - 1)
    omega, psi_b, ring = T(P.omega.ravel()), T(psi_b_h), T(P.psi_box)
    psibar = torch.zeros(1, dtype=torch.float64, device=dev)
    psi = torch.empty(NXY, dtype=torch.float64, device=dev)
    ux, uy = torch.empty_like(psi), torch.empty_like(psi)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream = torch.cuda.current_stream()

    def solve(prec, inner=None):
        return iim.iim_poisson_solve(geo, omega, psi_b, ring, None, psibar, psi, ux, uy,
                                     opts=iim.default_opts(prec=prec, rtol=RTOL, restart=args.restart,
                                                           inner_rtol=args.inner_rtol if inner is None else inner))

    if args.sweep:
        for prec in (iim.IIM_MIXED, iim.IIM_FP64):
            for inner in ((3e-3, 1e-3, 3e-4, 1e-4, 3e-5, 1e-5) if prec == iim.IIM_MIXED else (5e-12, 1e-11, 5e-11)):
                for _ in range(2):
                    solve(prec, inner)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(5):
                    st = solve(prec, inner)
                torch.cuda.synchronize()
                print(json.dumps({"prec": prec, "inner": inner, "ms": (time.perf_counter() - t0) / 5 * 1e3,
                                  "iters": st["iters"], "refinements": st["refinements"], "rel_res": st["rel_res"]}))
        return

    def timed(prec, k, warm):
        for _ in range(warm):
            solve(prec)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ms, stats = [], []
        for _ in range(k):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = solve(prec)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            stats.append(st)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        return ms, stats

    # ---- chosen form (timed region), with clocks sampled and launches counted
    with ClockSampler(local) as clk:
        l0 = iim.iim_launch_count()
        ms, stats = timed(iim.IIM_MIXED, args.steps, args.warmup)
        launches = iim.iim_launch_count() - l0
    total_ms = sum(ms)
    if ws > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = ws * args.steps / (total_ms * 1e-3)
    # ---- plain FP64 iteration (the comparator)
    k64 = max(3, args.steps // 5)
    ms64, stats64 = timed(iim.IIM_FP64, k64, max(3, args.warmup // 2))
    plain = k64 / (sum(ms64) * 1e-3)
    # ---- per-kernel timing of the same step (a second pass with CUDA events around kernels)
    kprof = min(args.steps, 10)
    iim.iim_profile_begin()
    for _ in range(kprof):
        flush.zero_()
        solve(iim.IIM_MIXED)
    kern = iim.iim_profile_end()
    kern.sort(key=lambda r: -r["ms"])
    tot_k = sum(r["ms"] for r in kern)
    peaks, src = measured_peaks()
    mem = [r for r in kern if r["bytes"] > 0]
    dom = mem[0] if mem else None
    roof = None
    if dom:
        per_launch_s = dom["ms"] * 1e-3 / dom["launches"]
        achieved = dom["bytes"] / dom["launches"] / per_launch_s / 1e9
        tr = NCU_TRAFFIC.get(dom["name"])
        traffic = tr["bytes_per_launch"] if tr and tr.get("source_hash") == kernel_source_hash() else None
        roof = {"bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "peak_source": src,
                "alg_bytes_per_launch": dom["bytes"] / dom["launches"], "avg_launch_us": per_launch_s * 1e6,
                "share_of_kernel_time": dom["ms"] / tot_k if tot_k else None}
    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        h_omega = torch.empty(NXY, dtype=torch.float64).pin_memory()
        h_omega.copy_(torch.from_numpy(np.ascontiguousarray(P.omega).ravel()))
        h_psib = torch.from_numpy(np.ascontiguousarray(psi_b_h)).pin_memory()
        h_ring = torch.from_numpy(np.ascontiguousarray(P.psi_box)).pin_memory()
        h_out = [torch.empty(NXY, dtype=torch.float64).pin_memory() for _ in range(3)]
        d_omega, d_psib, d_ring = torch.empty_like(omega), torch.empty_like(psi_b), torch.empty_like(ring)

        def e2e_step():
            d_omega.copy_(h_omega, non_blocking=True)
            d_psib.copy_(h_psib, non_blocking=True)
            d_ring.copy_(h_ring, non_blocking=True)
            iim.iim_poisson_solve(geo, d_omega, d_psib, d_ring, None, psibar, psi, ux, uy,
                                  opts=iim.default_opts(prec=iim.IIM_MIXED, rtol=RTOL))
            for h, d in zip(h_out, (psi, ux, uy)):
                h.copy_(d, non_blocking=True)

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        ems = []
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_step()
            b.record(stream)
            b.synchronize()
            ems.append(a.elapsed_time(b))
        e_total = sum(ems)
        if ws > 1:
            t = torch.tensor([e_total], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e_total = float(t.item())
        h2d = 8 * (NXY + psi_b.numel() + ring.numel())
        d2h = 8 * 3 * NXY
        e2e = {"value": ws * args.steps / (e_total * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.n)
    it = [s["iters"] for s in stats]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 transforms + f64 refinement", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "flushed before every timed step (256 MiB write, outside the events)",
                   "form": f"mixed: FP32 DST-I box solves inside FP64 iterative refinement, GMRES({args.restart}) FP64 Krylov",
                   "parallelism": f"replicas x{ws}"},
        "plain_fp64": {"value": plain, "unit": UNIT, "ms_per_step": sum(ms64) / k64,
                       "krylov_iters": statistics.mean(s["iters"] for s in stats64),
                       "final_rel_res": max(s["rel_res"] for s in stats64)},
        "speedup_vs_plain_fp64": value / plain / ws,
        "solver": {"krylov_iters": statistics.mean(it), "refinements": statistics.mean(s["refinements"] for s in stats),
                   "final_rel_res_max": max(s["rel_res"] for s in stats), "setup_s": t_setup,
                   "n_control": geo.n_control, "n_affected": geo.n_affected},
        "roofline": roof,
        "kernels": [{"name": r["name"], "launches_per_step": r["launches"] / kprof, "ms_per_step": r["ms"] / kprof,
                     "share": r["ms"] / tot_k if tot_k else None} for r in kern[:12]],
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line))
    geo.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
