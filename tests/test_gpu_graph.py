"""The whole solve as one device-driven graph (refinements, GMRES cycles and iterations decided by
control kernels on the device): from the second solve on a geometry it replaces the host-driven
loop, and it must give the same discrete result, iteration and refinement counts as the
host-driven first solve (the same kernels run in the same order)."""
import numpy as np
import pytest
import torch

import paper_2109_13628_gb300 as iim
from oracle import poisson as op
from paper_2109_13628_gb300 import inputs
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def _empty_box(n):
    g = inputs.square_grid(n)
    X, Y = g.nodes()
    w = inputs.gaussian_vortices(X, Y, [(0.3, -0.2)], [1.0], 0.3)
    return inputs.Problem(grid=g, phi=np.ones_like(X), regions=[], modes=[], omega=w[1:-1, 1:-1],
                          psi_box=inputs.box_ring(g, 0.5 * Y), psi_b_fn=lambda x, y, k: np.zeros_like(x),
                          psibar=np.zeros(0), gamma=None, exact=None)


CASES = {
    # restart 8 without preconditioner: several GMRES cycles, restart residuals on the device
    "restarts_fp64": (lambda: inputs.bicubic_bodies(128, seed=11, circulation=True),
                      dict(prec=iim.IIM_FP64, rtol=1e-12, restart=8, max_iter=4000), 0),
    # preconditioned mixed solve with a circulation body (capacitance correction in the graph)
    "precond_mixed_circulation": (lambda: inputs.c2_cylinder_flow(1024, 512),
                                  dict(prec=iim.IIM_MIXED, rtol=1e-10, precond=1), 1),
    # preconditioned with restart 2: every correction runs several cycles, so the one-block
    # GMRES start (restart residual) and back substitution run inside the cycle loop
    "restarts_precond_mixed": (lambda: inputs.bicubic_bodies(128, seed=11, circulation=True),
                               dict(prec=iim.IIM_MIXED, rtol=1e-11, restart=2, max_iter=4000, precond=1), 1),
    # no body: each refinement is one box solve
    "no_body": (lambda: _empty_box(128), dict(prec=iim.IIM_MIXED, rtol=1e-10), 0),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_graph_solve_matches_host_solve(case):
    make, kw, pc = CASES[case]
    P = make()
    geo = gu.setup(P)
    if pc:
        iim.iim_build_preconditioner(geo)
    gam = op.gamma_from_regions(P) + 0.05 if P.regions else None
    opts = iim.default_opts(**kw)
    first = gu.solve_opts(P, geo, gamma=gam, opts=opts, velocity=True)       # host-driven
    second = gu.solve_opts(P, geo, gamma=gam, opts=opts, velocity=True)      # builds and runs the graph
    n2 = iim.iim_launch_count()
    third = gu.solve_opts(P, geo, gamma=gam, opts=opts, velocity=True)       # the graph again
    n3 = iim.iim_launch_count()
    iim.iim_profile_begin()                                                 # profiling: host-driven
    gu.solve_opts(P, geo, gamma=gam, opts=opts, velocity=True)
    iim.iim_profile_end()
    n4 = iim.iim_launch_count()
    scale = np.abs(first["psi"]).max()
    for other in (second, third):
        assert np.abs(other["psi"] - first["psi"]).max() <= 1e-14 * scale
        assert np.abs(other["ux"] - first["ux"]).max() <= 1e-13 * max(np.abs(first["ux"]).max(), 1e-300)
        assert np.allclose(other["psibar"], first["psibar"], rtol=1e-13, atol=1e-14 * scale)
        for k in ("iters", "refinements", "status"):
            assert other["stats"][k] == first["stats"][k], (k, first["stats"], other["stats"])
        assert other["stats"]["rel_res"] == pytest.approx(first["stats"]["rel_res"], rel=1e-6, abs=1e-18)
        assert other["stats"]["circ_err_max"] <= 1e-12
    # the graph's kernels are counted per executed node, like the host path's launches (the graph
    # adds its loop-control kernels: a few per refinement, one per iteration)
    assert (n3 - n2) == pytest.approx(n4 - n3, rel=0.25, abs=8)
    geo.close()


def test_graph_rebuilt_for_new_arguments():
    """A solve into another output array after the graph was built writes there (the graph is
    keyed by its arguments)."""
    P = inputs.bicubic_bodies(64, seed=5, circulation=True)
    geo = gu.setup(P)
    gam = op.gamma_from_regions(P)
    opts = iim.default_opts(prec=iim.IIM_MIXED, rtol=1e-10)
    outs = [gu.solve_opts(P, geo, gamma=gam, opts=opts)["psi"] for _ in range(3)]   # host, graph, graph
    assert np.abs(outs[2] - outs[0]).max() <= 1e-14 * np.abs(outs[0]).max()
    # gu.solve_opts allocates new output tensors each call: every call above was a new key, so
    # the graph was rebuilt and still wrote the right array
    geo.close()
