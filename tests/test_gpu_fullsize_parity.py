"""Element-wise parity at the timed size: the single-cylinder workload at 1024^2 (1023^2
unknowns), the configuration the benchmark times, against the oracle's exact discrete solution
(the un-reduced sparse system of Sec. 4.2 solved directly).

FP64 mode must match to a relative L-infinity error of 1e-10, the mixed form (FP32 transforms in
FP64 refinement, dense Schur preconditioner) to 1e-8, both for psi and for the velocity.  The
mixed form is run through the batched entry point with several problems in flight, the launch
configuration of the benchmark, at the benchmark's stopping rule (residual 1e-10)."""
import numpy as np
import pytest
import torch

import paper_2109_13628_gb300 as iim
from oracle import poisson as op
from paper_2109_13628_gb300 import inputs
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1024():
    P = inputs.c1_cylinder(1024)
    S = op.Setup(P)
    ref, pb = op.solve_unreduced(S, psibar=np.zeros(1))
    ux, uy = op.velocity(S, ref, pb)
    fl = (P.phi >= 0)[1:-1, 1:-1]
    return P, ref[1:-1, 1:-1], ux, uy, fl


def rel(a, b, m):
    return np.abs(a - b)[m].max() / np.abs(b)[m].max()


def test_fp64_1024_elementwise(c1024):
    P, ref, ux, uy, fl = c1024
    geo = gu.setup(P)
    out = gu.solve(P, geo, prec=iim.IIM_FP64, rtol=1e-12, velocity=True)
    assert rel(out["psi"], ref, fl) < 1e-10
    assert rel(out["ux"], ux, fl) < 1e-10 and rel(out["uy"], uy, fl) < 1e-10
    geo.close()


@pytest.mark.parametrize("n_problems", [3])
def test_mixed_preconditioned_batch_1024_elementwise(c1024, n_problems):
    P, ref, ux, uy, fl = c1024
    geos = [gu.setup(P) for _ in range(n_problems)]
    cp = iim.iim_geometry_control_points(geos[0])
    psi_b = gu.T(P.psi_b_fn(cp["x"].cpu().numpy(), cp["y"].cpu().numpy(), None))
    om, ring = gu.T(P.omega.ravel()), gu.T(P.psi_box)
    NXY = P.omega.size
    psis = [torch.empty(NXY, dtype=torch.float64, device=gu.dev()) for _ in geos]
    uxs = [torch.empty_like(p) for p in psis]
    uys = [torch.empty_like(p) for p in psis]
    pbs = [torch.zeros(1, dtype=torch.float64, device=gu.dev()) for _ in geos]
    for geo in geos:
        iim.iim_build_preconditioner(geo)
    opts = iim.default_opts(prec=iim.IIM_MIXED, rtol=1e-10, restart=64, precond=1)
    for rep in range(2):   # first call: host-driven solves; second: the whole-solve graphs
        st, stats = iim.iim_poisson_solve_batched(geos, [om] * n_problems, [psi_b] * n_problems,
                                                  [ring] * n_problems, None, pbs, psis, uxs, uys, opts=opts,
                                                  n_streams=n_problems)
        assert st == iim.IIM_OK
        for k in range(n_problems):
            sh = ref.shape
            assert stats[k]["rel_res"] <= 1e-10
            assert rel(psis[k].cpu().numpy().reshape(sh), ref, fl) < 1e-8, (rep, k)
            assert rel(uxs[k].cpu().numpy().reshape(sh), ux, fl) < 1e-8
            assert rel(uys[k].cpu().numpy().reshape(sh), uy, fl) < 1e-8
    for geo in geos:
        geo.close()
