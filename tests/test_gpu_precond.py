"""Dense Schur-complement preconditioner: same discrete solution as the oracle, far fewer
Krylov iterations."""
import numpy as np
import pytest

import paper_2109_13628_gb300 as iim
from oracle import poisson as op
from paper_2109_13628_gb300 import inputs
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

TOL = {iim.IIM_FP64: 1e-10, iim.IIM_MIXED: 1e-8}


@pytest.mark.parametrize("n", [64, 256])
@pytest.mark.parametrize("prec", [iim.IIM_FP64, iim.IIM_MIXED])
def test_preconditioned_solve_matches_oracle(n, prec):
    P = inputs.bicubic_bodies(n, seed=n + 9, circulation=True)
    w = inputs.vortex_field(P.grid, 31, count=20, sigma=0.2)
    P.omega = np.where(P.phi >= 0, w, 0.0)[1:-1, 1:-1]
    S = op.Setup(P)
    gam = op.gamma_from_regions(P) + np.array([0.05, -0.1, 0.02])
    ref, pb_ref = op.solve_unreduced(S, gamma=gam)
    geo = gu.setup(P)
    ms = iim.iim_build_preconditioner(geo)
    assert ms > 0
    plain = gu.solve(P, geo, gamma=gam, prec=prec, rtol=1e-13)
    out = gu.solve_opts(P, geo, gamma=gam, opts=iim.default_opts(prec=prec, rtol=1e-13, max_iter=3000, precond=1))
    fl = (P.phi >= 0)[1:-1, 1:-1]
    err = np.abs(out["psi"] - ref[1:-1, 1:-1])[fl].max() / np.abs(ref).max()
    assert err < TOL[prec], (err, out["stats"])
    assert np.allclose(out["psibar"], pb_ref, rtol=TOL[prec], atol=TOL[prec] * np.abs(ref).max())
    assert out["stats"]["iters"] * 3 < plain["stats"]["iters"], (out["stats"], plain["stats"])
    # restart 2: many cycles per correction (restart residuals, updates inside the cycle loop)
    short = gu.solve_opts(P, geo, gamma=gam, opts=iim.default_opts(prec=prec, rtol=1e-13, max_iter=3000, restart=2,
                                                                   precond=1))
    err2 = np.abs(short["psi"] - ref[1:-1, 1:-1])[fl].max() / np.abs(ref).max()
    assert err2 < TOL[prec], (err2, short["stats"])
    geo.close()


def test_preconditioned_c1_1024_to_1e10():
    P = inputs.c1_cylinder(1024)
    S = op.Setup(P)
    geo = gu.setup(P)
    out = gu.solve_opts(P, geo, opts=iim.default_opts(prec=iim.IIM_MIXED, rtol=1e-10, precond=1))
    nodes = gu.nodes_from_interior(P, out["psi"])
    assert op.residual(S, nodes, out["psibar"]) < 1e-10
    assert out["stats"]["iters"] <= 16, out["stats"]   # plain GMRES needs about 100 here
    assert out["stats"]["iters"] < 20, out["stats"]
    geo.close()


@pytest.mark.parametrize("prec", [iim.IIM_FP64, iim.IIM_MIXED])
def test_direct_corrections_match_oracle(prec):
    """precond = 2: every correction is one application of the dense inverse (no Krylov
    iterations unless the fallback to GMRES fires); the result is the same discrete solution."""
    n = 128
    P = inputs.bicubic_bodies(n, seed=n + 9, circulation=True)
    w = inputs.vortex_field(P.grid, 31, count=20, sigma=0.2)
    P.omega = np.where(P.phi >= 0, w, 0.0)[1:-1, 1:-1]
    S = op.Setup(P)
    gam = op.gamma_from_regions(P) + np.array([0.05, -0.1, 0.02])
    ref, pb_ref = op.solve_unreduced(S, gamma=gam)
    geo = gu.setup(P)
    out = gu.solve_opts(P, geo, gamma=gam, opts=iim.default_opts(prec=prec, rtol=1e-13, max_iter=3000, precond=2))
    fl = (P.phi >= 0)[1:-1, 1:-1]
    err = np.abs(out["psi"] - ref[1:-1, 1:-1])[fl].max() / np.abs(ref).max()
    assert err < TOL[prec], (err, out["stats"])
    assert out["stats"]["rel_res"] <= 1e-13
    if not out["stats"]["fallback"] & 2:
        assert out["stats"]["iters"] == 0
    geo.close()


@pytest.mark.parametrize("n", [64, 256])
@pytest.mark.parametrize("prec", [iim.IIM_FP64, iim.IIM_MIXED])
def test_dense_inner_operator_matches_oracle(n, prec):
    """precond = 3: the inner Krylov operator is the dense FP32 Schur matrix (formed with the
    preconditioner) instead of the transforms; the FP64 un-reduced residual still decides
    convergence, so the solution is the same discrete solution within the stated tolerances,
    with restart 64 and with restart 2 (restart residuals through the dense operator), and the
    graph-driven solve equals the host-driven one bit for bit."""
    P = inputs.bicubic_bodies(n, seed=n + 9, circulation=True)
    w = inputs.vortex_field(P.grid, 31, count=20, sigma=0.2)
    P.omega = np.where(P.phi >= 0, w, 0.0)[1:-1, 1:-1]
    S = op.Setup(P)
    gam = op.gamma_from_regions(P) + np.array([0.05, -0.1, 0.02])
    ref, pb_ref = op.solve_unreduced(S, gamma=gam)
    geo = gu.setup(P)
    fl = (P.phi >= 0)[1:-1, 1:-1]
    for restart in (64, 2):
        opts = iim.default_opts(prec=prec, rtol=1e-13, max_iter=3000, restart=restart, precond=3)
        first = gu.solve_opts(P, geo, gamma=gam, opts=opts)     # host-driven (first solve with these options)
        again = gu.solve_opts(P, geo, gamma=gam, opts=opts)     # whole-solve graph
        for out in (first, again):
            err = np.abs(out["psi"] - ref[1:-1, 1:-1])[fl].max() / np.abs(ref).max()
            assert err < TOL[prec], (restart, err, out["stats"])
            assert np.allclose(out["psibar"], pb_ref, rtol=TOL[prec], atol=TOL[prec] * np.abs(ref).max())
            assert out["stats"]["rel_res"] <= 1e-13
        assert np.array_equal(first["psi"], again["psi"])
        assert first["stats"]["iters"] == again["stats"]["iters"]
    geo.close()
