"""Batched solves: every problem of a mixed-size batch gets exactly the result of its own
single solve, and matches the oracle."""
import numpy as np
import pytest
import torch

import paper_2109_13628_gb300 as iim
from oracle import poisson as op
from paper_2109_13628_gb300 import autotune, inputs
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def build_batch(problems):
    geos, args = [], {k: [] for k in ("omega", "psi_b", "gamma", "psibar", "psi")}
    kept = []
    for P in problems:
        try:
            geo = gu.setup(P)
        except iim.IIMError:
            continue                      # under-resolved draw: skipped like in the benchmark
        kept.append(P)
        geos.append(geo)
        args["omega"].append(gu.T(P.omega.ravel()))
        args["psi_b"].append(gu.T(gu.psi_b_for(P, geo)))
        args["gamma"].append(gu.T(op.gamma_from_regions(P)))
        args["psibar"].append(torch.zeros(len(P.regions), dtype=torch.float64, device=gu.dev()))
        args["psi"].append(torch.empty(P.omega.size, dtype=torch.float64, device=gu.dev()))
    return kept, geos, args


@pytest.mark.parametrize("precond", [0, 1])
def test_batched_equals_single_solves_and_oracle(precond):
    problems = inputs.batched_c4(count=10, seed=5, sizes=(64, 128, 256))
    kept, geos, a = build_batch(problems)
    assert len(kept) >= 6
    opts = iim.default_opts(prec=iim.IIM_MIXED, rtol=1e-12, precond=precond)
    st, stats = iim.iim_poisson_solve_batched(geos, a["omega"], a["psi_b"], None, a["gamma"], a["psibar"], a["psi"],
                                              opts=opts, n_streams=4)
    assert st == iim.IIM_OK
    for k, (P, geo) in enumerate(zip(kept, geos)):
        single = torch.empty_like(a["psi"][k])
        pb = torch.zeros_like(a["psibar"][k])
        iim.iim_poisson_solve(geo, a["omega"][k], a["psi_b"][k], None, a["gamma"][k], pb, single, opts=opts)
        assert torch.equal(single, a["psi"][k])
        assert stats[k]["rel_res"] < 1e-12
    # oracle parity on the two smallest problems
    for k in np.argsort([P.grid.nx for P in kept])[:2]:
        P = kept[k]
        ref, pb_ref = op.solve_unreduced(op.Setup(P), gamma=op.gamma_from_regions(P))
        out = a["psi"][k].cpu().numpy().reshape(P.omega.shape)
        fl = (P.phi >= 0)[1:-1, 1:-1]
        assert np.abs(out - ref[1:-1, 1:-1])[fl].max() < 1e-8 * np.abs(ref).max()
    for g in geos:
        g.close()


def test_autotuner_picks_supported_tiles():
    problems = inputs.batched_c4(count=4, seed=7, sizes=(128, 256))
    kept, geos, a = build_batch(problems)
    opts = iim.default_opts(prec=iim.IIM_MIXED, rtol=1e-10)

    def solve_one(k):
        pb = torch.zeros_like(a["psibar"][k])
        iim.iim_poisson_solve(geos[k], a["omega"][k], a["psi_b"][k], None, a["gamma"][k], pb, a["psi"][k], opts=opts)

    best = autotune.tune_tiles(geos, solve_one)
    assert set(best.values()) <= {2, 4, 8}
    n_best, times = autotune.tune_streams(lambda c: iim.iim_poisson_solve_batched(
        geos, a["omega"], a["psi_b"], None, a["gamma"], a["psibar"], a["psi"], opts=opts, n_streams=c), (1, 2, 4))
    assert n_best in (1, 2, 4) and all(t > 0 for t in times.values())
    for g in geos:
        g.close()


@pytest.mark.parametrize("precond", [0, 1])
def test_batched_host_buffers_equal_device_batch(precond):
    """iim_poisson_solve_batched_host on host tensors gives exactly the device batch's results
    (psi, u, psibar), on a first call (host-driven solves) and on later calls (whole-solve
    graphs); outputs in pinned memory are written there by the last kernel, pageable outputs
    are staged and copied -- both paths are exercised."""
    problems = inputs.batched_c4(count=8, seed=5, sizes=(64, 128, 256))
    kept, geos, a = build_batch(problems)
    opts = iim.default_opts(prec=iim.IIM_MIXED, rtol=1e-11, precond=precond)
    ux = [torch.empty_like(t) for t in a["psi"]]
    uy = [torch.empty_like(t) for t in a["psi"]]
    st, ref_stats = iim.iim_poisson_solve_batched(geos, a["omega"], a["psi_b"], None, a["gamma"], a["psibar"],
                                                  a["psi"], ux, uy, opts=opts, n_streams=3)
    assert st == iim.IIM_OK
    pin = lambda t: t.cpu().pin_memory()
    h_om = [pin(t) for t in a["omega"]]
    h_pb = [pin(t) for t in a["psi_b"]]
    h_gm = [pin(t) for t in a["gamma"]]
    for call in range(4):
        pinned = call % 2 == 0
        out = lambda t: (torch.full((t.numel(),), np.nan, dtype=torch.float64).pin_memory() if pinned
                         else torch.full((t.numel(),), np.nan, dtype=torch.float64))
        h_pbar = [torch.zeros(t.numel(), dtype=torch.float64).pin_memory() for t in a["psibar"]]
        h_psi = [out(t) for t in a["psi"]]
        h_ux = [out(t) for t in a["psi"]]
        h_uy = [out(t) for t in a["psi"]]
        st, stats = iim.iim_poisson_solve_batched_host(geos, h_om, h_pb, None, h_gm, h_pbar, h_psi, h_ux, h_uy,
                                                       opts=opts, n_streams=3)
        assert st == iim.IIM_OK
        for k in range(len(kept)):
            assert torch.equal(h_psi[k], a["psi"][k].cpu()), (call, k)
            assert torch.equal(h_ux[k], ux[k].cpu()), (call, k)
            assert torch.equal(h_uy[k], uy[k].cpu()), (call, k)
            assert torch.equal(h_pbar[k], a["psibar"][k].cpu())
            assert stats[k]["iters"] == ref_stats[k]["iters"]
    for g in geos:
        g.close()


def test_empty_and_single_problem_batches():
    """n = 0 is a no-op in both batched calls; a batch of one equals the single solve."""
    opts = iim.default_opts(prec=iim.IIM_MIXED, rtol=1e-11)
    st, stats = iim.iim_poisson_solve_batched([], [], [], None, None, [], [], opts=opts, n_streams=4)
    assert st == iim.IIM_OK and stats == []
    st, stats = iim.iim_poisson_solve_batched_host([], [], [], None, None, [], [], opts=opts, n_streams=4)
    assert st == iim.IIM_OK and stats == []
    kept, geos, a = build_batch(inputs.batched_c4(count=4, seed=5, sizes=(128,)))
    assert len(kept) >= 1
    one = lambda k: [a[k][0]]
    st, stats = iim.iim_poisson_solve_batched(geos[:1], one("omega"), one("psi_b"), None, one("gamma"), one("psibar"),
                                              one("psi"), opts=opts, n_streams=4)
    assert st == iim.IIM_OK and len(stats) == 1
    psi1 = torch.empty_like(a["psi"][0])
    pb1 = torch.zeros_like(a["psibar"][0])
    s1 = iim.iim_poisson_solve(geos[0], a["omega"][0], a["psi_b"][0], None, a["gamma"][0], pb1, psi1, opts=opts)
    assert torch.equal(psi1, a["psi"][0]) and s1["iters"] == stats[0]["iters"]
    for g in geos:
        g.close()


@pytest.mark.parametrize("prec,precond", [(iim.IIM_FP64, 1), (iim.IIM_MIXED, 1), (iim.IIM_MIXED, 3)])
def test_lockstep_groups_equal_single_solves(prec, precond):
    """From the second batched call on, the problems of each grid size advance as one lockstep
    group (one launch per step for the whole group, loops decided on the device).  Every problem
    gets exactly its single solve's psi, u, psibar, iteration and refinement counts; lockstep
    issues fewer launches than one whole-solve graph per problem; with the per-kernel profiler
    on, the same groups run host-driven, give the same results, and the profile holds the
    batched kernels."""
    problems = inputs.batched_c4(count=10, seed=5, sizes=(64, 128, 256))
    kept, geos, a = build_batch(problems)
    opts = iim.default_opts(prec=prec, rtol=1e-11, precond=precond)
    ux = [torch.empty_like(t) for t in a["psi"]]
    uy = [torch.empty_like(t) for t in a["psi"]]

    def batch():
        for t in a["psi"] + ux + uy:
            t.fill_(float("nan"))
        for t in a["psibar"]:
            t.zero_()
        before = iim.iim_launch_count()
        st, stats = iim.iim_poisson_solve_batched(geos, a["omega"], a["psi_b"], None, a["gamma"], a["psibar"],
                                                  a["psi"], ux, uy, opts=opts, n_streams=3)
        assert st == iim.IIM_OK
        return ([t.clone() for t in a["psi"]], [t.clone() for t in ux], [t.clone() for t in uy],
                [t.clone() for t in a["psibar"]], stats, iim.iim_launch_count() - before)

    batch()                                   # first solves: host-driven, per problem
    prev = iim.iim_set_lockstep(0)
    per_problem = batch()                     # one whole-solve graph per problem
    iim.iim_set_lockstep(2)
    pairs = batch()                           # lockstep groups of two, concurrent
    iim.iim_set_lockstep(64)
    lock = batch()                            # one lockstep group per grid size
    iim.iim_profile_begin()
    hosted = batch()                          # lockstep, host-driven under the profiler
    prof = iim.iim_profile_end()
    iim.iim_set_lockstep(prev)
    sizes = [P.grid.nx for P in kept]
    assert max(sizes.count(n) for n in set(sizes)) >= 2     # at least one real group
    for k, (P, geo) in enumerate(zip(kept, geos)):
        psi1, ux1, uy1 = (torch.empty_like(a["psi"][k]) for _ in range(3))
        pb1 = torch.zeros_like(a["psibar"][k])
        s1 = iim.iim_poisson_solve(geo, a["omega"][k], a["psi_b"][k], None, a["gamma"][k], pb1, psi1, ux1, uy1,
                                   opts=opts)
        for run in (per_problem, pairs, lock, hosted):
            assert torch.equal(run[0][k], psi1) and torch.equal(run[1][k], ux1) and torch.equal(run[2][k], uy1), k
            assert torch.equal(run[3][k], pb1)
            assert run[4][k]["iters"] == s1["iters"] and run[4][k]["refinements"] == s1["refinements"]
            assert run[4][k]["rel_res"] == s1["rel_res"] and run[4][k]["rel_res"] < 1e-11
    assert lock[5] < per_problem[5]
    names = {r["name"] for r in prof}
    assert ("ls_tri_cols_f64" if prec == iim.IIM_FP64 else "ls_tri_cols_f32") in names   # default column pass
    assert ("ls_dense_schur_matvec" in names) == (precond == 3)
    assert "ls_gmres_arnoldi" in names and "ls_residual_f64" in names
    for g in geos:
        g.close()
