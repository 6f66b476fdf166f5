"""GPU parity of the transport step (vorticity BC, transport RHS, Kelvin, RK3) against the
oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import paper_2109_13628_gb300 as iim
from oracle import poisson as op
from oracle import transport as tr
from paper_2109_13628_gb300 import inputs
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def two_body(n):
    g = inputs.square_grid(n)
    X, Y = g.nodes()
    a = inputs.phi_circle(X, Y, -0.8, -0.7, 0.45)
    b = inputs.phi_star(X, Y, 0.7, 0.6, 0.45, 0.08, 4)
    phi = inputs.union(a, b)
    return inputs.Problem(grid=g, phi=phi, regions=[inputs.region_around(g, a), inputs.region_around(g, b)],
                          modes=[1, 1], omega=np.zeros((n - 1, n - 1)), psi_box=np.zeros(4 * n),
                          psi_b_fn=lambda x, y, k: np.zeros_like(x), psibar=np.zeros(2), gamma=None, exact=None)


@pytest.mark.parametrize("n", [64, 128])
@pytest.mark.parametrize("Uinf", [(0.0, 0.0), (0.8, -0.3)])
def test_transport_rhs_matches_oracle(n, Uinf):
    P = two_body(n)
    S = op.Setup(P)
    T = tr.TransportSetup(S)
    g = P.grid
    fl = (P.phi >= 0)[1:-1, 1:-1]
    w = np.where(fl, inputs.vortex_field(g, 12, count=15, sigma=0.25)[1:-1, 1:-1], 0)
    psi, pb = op.solve_unreduced(S, omega=w, gamma=op.gamma_from_regions(P) + 0.1)
    ux, uy = op.velocity(S, psi, pb)
    ux = ux + Uinf[0] * fl
    uy = uy + Uinf[1] * fl
    ncp = S.geo["cp"]["t"].size
    rng = np.random.default_rng(n)
    u_b = (0.1 * rng.normal(size=ncp), 0.1 * rng.normal(size=ncp))
    nu = 0.004
    rhs, Fx, Fy, wb = tr.transport_rhs(T, w, ux, uy, u_b, Uinf, nu)
    dG = tr.kelvin_rhs(S, Fx, Fy)
    geo = gu.setup(P)
    NXY = (n - 1) ** 2
    out = torch.empty(NXY, dtype=torch.float64, device=gu.dev())
    wb_g = torch.empty(geo.n_control, dtype=torch.float64, device=gu.dev())
    dg_g = torch.empty(2, dtype=torch.float64, device=gu.dev())
    iim.iim_transport_rhs(geo, gu.T(w.ravel()), gu.T(ux.ravel()), gu.T(uy.ravel()), gu.T(np.concatenate(u_b)), Uinf, nu,
                          out, omega_b_out=wb_g, dgamma_out=dg_g)
    wbg = wb_g.cpu().numpy()
    assert np.abs(wbg - wb).max() < 1e-11 * max(1.0, np.abs(wb).max())
    r = out.cpu().numpy().reshape(n - 1, n - 1)
    assert np.abs(r - rhs).max() < 1e-11 * np.abs(rhs).max()
    assert np.allclose(dg_g.cpu().numpy(), dG, rtol=1e-11, atol=1e-13)
    geo.close()


def test_transport_rhs_polynomial_exactness_full_size():
    """Any size: bilinear vorticity and linear divergence-free velocity are transported exactly."""
    P = inputs.c2_cylinder_flow(1024, 512)
    geo = gu.setup(P)
    Xi, Yi = P.grid.interior()
    a, b, c, d = 0.7, -0.4, 0.3, 0.9
    al, be, ga, de = 0.2, 1.1, -0.6, 0.5
    fl = (P.phi >= 0)[1:-1, 1:-1]
    ux, uy = np.where(fl, a + b * Yi, 0), np.where(fl, c + d * Xi, 0)
    w = np.where(fl, al + be * Xi + ga * Yi + de * Xi * Yi, 0)
    cp = {k: v.cpu().numpy() for k, v in iim.iim_geometry_control_points(geo).items()}
    u_b = np.concatenate([a + b * cp["y"], c + d * cp["x"]])
    out = torch.empty(w.size, dtype=torch.float64, device=gu.dev())
    wb_g = torch.empty(geo.n_control, dtype=torch.float64, device=gu.dev())
    iim.iim_transport_rhs(geo, gu.T(w.ravel()), gu.T(ux.ravel()), gu.T(uy.ravel()), gu.T(u_b), (0.0, 0.0), 0.005, out,
                          omega_b_out=wb_g)
    # omega_b of this linear velocity is curl u = d - b exactly
    assert np.abs(wb_g.cpu().numpy() - (d - b)).max() < 1e-9
    # with the wall vorticity of the bilinear field prescribed, the RHS is exact near the body
    wb_exact = al + be * cp["x"] + ga * cp["y"] + de * cp["x"] * cp["y"]
    iim.iim_transport_rhs(geo, gu.T(w.ravel()), gu.T(ux.ravel()), gu.T(uy.ravel()), gu.T(u_b), (0.0, 0.0), 0.005, out,
                          omega_b_in=gu.T(wb_exact))
    r = out.cpu().numpy().reshape(w.shape)
    exact = -(ux * (be + de * Yi) + uy * (ga + de * Xi))
    keep = np.zeros_like(fl)
    keep[3:-3, 3:-3] = True
    m = fl & keep
    assert np.abs(r - exact)[m].max() < 1e-9 * np.abs(exact).max()
    geo.close()


@pytest.mark.parametrize("prec", [iim.IIM_FP64, iim.IIM_MIXED])
def test_rk3_step_matches_oracle_c2_small(prec):
    P = inputs.c2_cylinder_flow(128, 64)
    S = op.Setup(P)
    T = tr.TransportSetup(S)
    gam0 = op.gamma_from_regions(P)
    ncp = S.geo["cp"]["t"].size
    zero_b = (np.zeros(ncp), np.zeros(ncp))
    nu, Uinf, cst = 0.005, (1.0, 0.0), 0.5
    w1, g1, dt, pb = tr.rk3_step(T, P.omega, gam0, zero_b, Uinf, nu, cst)
    geo = gu.setup(P)
    w = gu.T(P.omega.ravel())
    gam = gu.T(gam0)
    pbar = torch.zeros(1, dtype=torch.float64, device=gu.dev())
    dt_g, stats, _ = iim.iim_rk3_step(geo, w, gam, pbar, None, None, gu.T(P.psi_box), Uinf, nu, cst,
                                       opts=iim.default_opts(prec=prec, rtol=1e-13))
    tol = 1e-10 if prec == iim.IIM_FP64 else 1e-8
    assert abs(dt_g - dt) < 1e-12 * dt
    wg = w.cpu().numpy().reshape(P.omega.shape)
    assert np.abs(wg - w1).max() < tol * np.abs(w1).max()
    assert abs(gam.cpu().numpy()[0] - g1[0]) < tol * max(1.0, abs(g1[0]))
    geo.close()


def test_rk3_kelvin_invariant_on_gpu():
    """Gamma + h^2 sum of omega outside R is conserved by a GPU RK3 step when no vorticity
    leaves the box (discrete Kelvin theorem, Sec. 5.1)."""
    P = two_body(128)
    g = P.grid
    X, Y = g.nodes()
    fl = (P.phi >= 0)[1:-1, 1:-1]
    w0 = np.where(fl, inputs.gaussian_vortices(X, Y, [(0.4, -0.6), (-0.6, 0.7)], [1.0, -0.7], 0.12)[1:-1, 1:-1], 0)
    gam0 = op.gamma_from_regions(inputs.Problem(**{**P.__dict__, "omega": w0})) + np.array([0.02, -0.03])
    geo = gu.setup(P)
    w = gu.T(w0.ravel())
    gam = gu.T(gam0)
    pbar = torch.zeros(2, dtype=torch.float64, device=gu.dev())
    dt, stats, _ = iim.iim_rk3_step(geo, w, gam, pbar, None, None, None, (0.0, 0.0), 0.01, 0.5,
                                     opts=iim.default_opts(prec=iim.IIM_MIXED, rtol=1e-12))
    h = g.h
    inside = np.zeros_like(fl)
    for (lx, rx, ly, ry) in P.regions:
        inside[ly - 1:ry, lx - 1:rx] = True
    w1 = w.cpu().numpy().reshape(w0.shape)
    before = gam0.sum() + h * h * w0[~inside].sum()
    after = gam.cpu().numpy().sum() + h * h * w1[~inside].sum()
    assert abs(after - before) < 1e-12
    assert np.abs(w1[~fl]).max() == 0.0
    geo.close()


def test_rk3_third_order_in_time_on_gpu():
    """The GPU step under temporal refinement at fixed h: a weak Gaussian vortex carried by the
    free stream (1, 0.3) through an empty 128^2 box, to t = 0.04 with dt = 0.02, 0.01, 0.005
    against dt = 0.0025 (FP64 solves to 1e-12); the error falls by about 2^3 per halving."""
    n = 128
    g = inputs.square_grid(n)
    X, Y = g.nodes()
    P = inputs.Problem(grid=g, phi=np.ones_like(X), regions=[], modes=[], omega=np.zeros((n - 1, n - 1)),
                       psi_box=inputs.box_ring(g, 1.0 * Y - 0.3 * X), psi_b_fn=lambda x, y, k: np.zeros_like(x),
                       psibar=np.zeros(0), gamma=None, exact=None)
    geo = gu.setup(P)
    w0 = (0.05 * inputs.gaussian_vortices(X, Y, [(-0.5, -0.2)], [1.0], 0.3))[1:-1, 1:-1]
    ring = gu.T(P.psi_box)
    opts = iim.default_opts(prec=iim.IIM_FP64, rtol=1e-12)

    def run(dt, steps):
        w = gu.T(w0.ravel())
        for _ in range(steps):
            iim.iim_rk3_step(geo, w, None, None, None, None, ring, (1.0, 0.3), 0.002, 0.5, dt=dt, opts=opts)
        return w.cpu().numpy()

    ref = run(0.0025, 16)
    errs = [np.abs(run(dt, steps) - ref).max() for dt, steps in ((0.02, 2), (0.01, 4), (0.005, 8))]
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 2.6, (errs, orders)
    geo.close()


def test_checkpoint_resume_repeats_next_step_bitwise(tmp_path):
    """The integration state (Sec. 5.5: omega, Gamma_k, t; psibar_k kept as well) saved after
    one RK3 step and loaded into a fresh geometry repeats the original run's next step bit for
    bit."""
    from paper_2109_13628_gb300 import checkpoint
    P = inputs.c2_cylinder_flow(128, 64)
    opts = iim.default_opts(prec=iim.IIM_MIXED, rtol=1e-11)
    nu, Uinf, cst = 0.005, (1.0, 0.0), 0.5
    ring = gu.T(P.psi_box)
    geo = gu.setup(P)
    w, gam = gu.T(P.omega.ravel()), gu.T(op.gamma_from_regions(P))
    pbar = torch.zeros(1, dtype=torch.float64, device=gu.dev())
    dt1, _, _ = iim.iim_rk3_step(geo, w, gam, pbar, None, None, ring, Uinf, nu, cst, opts=opts)
    path = str(tmp_path / "flow")
    checkpoint.save(path, {"omega": w, "gamma": gam, "psibar": pbar}, t=dt1, step=1, grid=P.grid, meta={"nu": nu})
    dt2, _, _ = iim.iim_rk3_step(geo, w, gam, pbar, None, None, ring, Uinf, nu, cst, opts=opts)
    geo.close()
    state, hdr = checkpoint.load(path, device=gu.dev())
    assert hdr["step"] == 1 and hdr["t"] == dt1
    geo2 = gu.setup(P)
    w2, gam2, pbar2 = state["omega"], state["gamma"], state["psibar"]
    dt2b, _, _ = iim.iim_rk3_step(geo2, w2, gam2, pbar2, None, None, ring, Uinf, nu, cst, opts=opts)
    assert dt2b == dt2
    assert torch.equal(w2, w) and torch.equal(gam2, gam) and torch.equal(pbar2, pbar)
    geo2.close()
