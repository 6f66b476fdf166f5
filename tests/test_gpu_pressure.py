"""GPU parity of the total-pressure problem (Sec. 5.4) and of the Neumann ghost stencils
(Sec. 2.1) against the oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import paper_2109_13628_gb300 as iim
from oracle import poisson as op
from oracle import pressure as pr
from oracle import transport as tr
from paper_2109_13628_gb300 import inputs
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def _neumann_data_at(cp, grad_fn):
    """d . grad f at the control points of a device geometry (d from the solid end to the fluid)."""
    x, y = cp["x"].cpu().numpy(), cp["y"].cpu().numpy()
    gx, gy = grad_fn(x, y)
    return gx, gy


def _data_oracle(S, grad_fn):
    cps = S.geo["cp"]
    gx, gy = grad_fn(cps["x"], cps["y"])
    return (cps["fi"] - cps["si"]) * gx + (cps["fj"] - cps["sj"]) * gy


def _bicubic_grad(c):
    def grad(x, y):
        gx, gy = np.zeros_like(x), np.zeros_like(x)
        for a in range(4):
            for b in range(4):
                if a:
                    gx = gx + c[a, b] * a * x ** (a - 1) * y ** b
                if b:
                    gy = gy + c[a, b] * b * x ** a * y ** (b - 1)
        return gx, gy
    return grad


def _neumann_geometry(P):
    geo = gu.setup(P)
    iim.iim_geometry_set_wall_condition(geo, 1)
    return geo


def _solve(P, geo, f, data, ring, prec, precond=0, rtol=1e-12):
    NXY = (P.grid.nx - 1) * (P.grid.ny - 1)
    H = torch.empty(NXY, dtype=torch.float64, device=gu.dev())
    opts = iim.default_opts(prec=prec, rtol=rtol, precond=precond, restart=64, max_iter=3000)
    st = iim.iim_poisson_solve(geo, gu.T(np.ascontiguousarray(f).ravel()), gu.T(data), gu.T(ring), None, None, H,
                               opts=opts)
    return H.cpu().numpy().reshape(P.grid.ny - 1, P.grid.nx - 1), st


@pytest.mark.parametrize("n", [64, 256])
@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_precond", "mixed_dense_op"])
def test_neumann_solve_exact_for_bicubic_fields(n, mode):
    """Around a circle, an ellipse and a nonconvex star, the discrete Neumann solution of a bicubic
    field is the field itself; the GPU reaches it in every mode."""
    P = inputs.bicubic_bodies(n, seed=1, circulation=False)
    c = inputs.bicubic_coeffs(1)
    geo = _neumann_geometry(P)
    cp = iim.iim_geometry_control_points(geo)
    S = op.Setup(P, wall="neumann", wall_data=np.zeros(1))
    data = _data_oracle(S, _bicubic_grad(c))
    # the device's control points are the oracle's, in the same canonical order
    assert np.allclose(cp["x"].cpu().numpy(), S.geo["cp"]["x"], atol=1e-12)
    prec, pc = {"fp64": (iim.IIM_FP64, 0), "mixed": (iim.IIM_MIXED, 0), "mixed_precond": (iim.IIM_MIXED, 1),
                "mixed_dense_op": (iim.IIM_MIXED, 3)}[mode]
    H, st = _solve(P, geo, P.omega, data, P.psi_box, prec, pc, rtol=1e-12 if prec == iim.IIM_FP64 else 1e-10)
    fl = P.phi[1:-1, 1:-1] >= 0
    scale = np.abs(P.exact).max()
    tol = 1e-10 if prec == iim.IIM_FP64 else 1e-8
    assert np.abs(np.where(fl, H - P.exact[1:-1, 1:-1], 0.0)).max() < tol * scale, st
    assert np.all(H[~fl] == 0.0)
    geo.close()


@pytest.mark.parametrize("prec", [iim.IIM_FP64, iim.IIM_MIXED])
def test_neumann_solve_matches_oracle_elementwise(prec):
    """A smooth manufactured field on the single cylinder: the GPU solution equals the oracle's
    un-reduced sparse solution element by element (1e-10 FP64, 1e-8 mixed, relative to max |H|)."""
    n = 128
    P = inputs.c1_cylinder(n)
    X, Y = P.grid.nodes()
    Hx = np.sin(1.3 * X + 0.4) * np.cos(0.9 * Y)
    P.omega = np.ascontiguousarray(np.where(P.phi >= 0, 2.5 * Hx, 0.0)[1:-1, 1:-1])
    P.psi_box = inputs.box_ring(P.grid, Hx)
    S0 = op.Setup(P, wall="neumann", wall_data=np.zeros(1))
    data = _data_oracle(S0, lambda x, y: (1.3 * np.cos(1.3 * x + 0.4) * np.cos(0.9 * y),
                                          -0.9 * np.sin(1.3 * x + 0.4) * np.sin(0.9 * y)))
    S = op.Setup(P, wall="neumann", wall_data=data)
    ref, _ = op.solve_unreduced(S, psibar=np.zeros(1))
    geo = _neumann_geometry(P)
    H, st = _solve(P, geo, P.omega, data, P.psi_box, prec, 1 if prec == iim.IIM_MIXED else 0,
                   rtol=1e-12 if prec == iim.IIM_FP64 else 1e-10)
    tol = 1e-10 if prec == iim.IIM_FP64 else 1e-8
    fl = P.phi[1:-1, 1:-1] >= 0
    assert np.abs(np.where(fl, H - ref[1:-1, 1:-1], 0.0)).max() < tol * np.abs(ref).max(), st
    geo.close()


def test_wall_condition_switch_back_is_bit_exact():
    """Dirichlet -> Neumann -> Dirichlet restores the stencils exactly: the Dirichlet solve after the
    round trip equals the one before, bit for bit."""
    P = inputs.bicubic_bodies(64, seed=0, circulation=False)
    geo = gu.setup(P)
    a = gu.solve(P, geo, psibar=P.psibar)["psi"]
    iim.iim_geometry_set_wall_condition(geo, 1)
    iim.iim_geometry_set_wall_condition(geo, 0)
    b = gu.solve(P, geo, psibar=P.psibar)["psi"]
    assert np.array_equal(a, b)
    geo.close()


def test_wall_condition_rejects_circulation_bodies():
    P = inputs.bicubic_bodies(64, seed=0, circulation=True)
    geo = gu.setup(P)
    with pytest.raises(iim.IIMError):
        iim.iim_geometry_set_wall_condition(geo, 1)
    with pytest.raises(iim.IIMError):
        iim.iim_geometry_set_wall_condition(geo, 2)
    geo.close()


def _flow_snapshot(n, Uinf=(0.6, -0.2)):
    """A cylinder and a nonconvex star with stationary no-slip walls, a seeded vortex field and the
    velocity of its IIM solve plus a free stream (the flow solver's form of the problem)."""
    g = inputs.square_grid(n)
    X, Y = g.nodes()
    a = inputs.phi_circle(X, Y, -0.8, -0.7, 0.45)
    b = inputs.phi_star(X, Y, 0.7, 0.6, 0.45, 0.08, 4)
    phi = inputs.union(a, b)
    P = inputs.Problem(grid=g, phi=phi, regions=[inputs.region_around(g, a), inputs.region_around(g, b)],
                       modes=[0, 0], omega=np.zeros((n - 1, n - 1)), psi_box=np.zeros(4 * n),
                       psi_b_fn=lambda x, y, k: np.zeros_like(x), psibar=np.zeros(2), gamma=None, exact=None)
    S = op.Setup(P)
    fl = (phi >= 0)[1:-1, 1:-1]
    w = np.where(fl, inputs.vortex_field(g, 21, count=15, sigma=0.25)[1:-1, 1:-1], 0.0)
    psi, pb = op.solve_unreduced(S, omega=w, psibar=np.array([0.05, -0.03]))
    ux, uy = op.velocity(S, psi, pb)
    return P, S, w, ux + Uinf[0] * fl, uy + Uinf[1] * fl, Uinf


@pytest.mark.parametrize("n", [64, 128])
def test_total_pressure_problem_matches_oracle(n):
    P, S, w, ux, uy, Uinf = _flow_snapshot(n)
    T = tr.TransportSetup(S)
    ncp = S.geo["cp"]["t"].size
    nu = 0.004
    f, wb = pr.pressure_rhs(T, w, ux, uy, (np.zeros(ncp), np.zeros(ncp)), Uinf)
    data = pr.wall_data(T, w, wb, nu)
    geo = _neumann_geometry(P)
    NXY = (n - 1) ** 2
    f_g = torch.empty(NXY, dtype=torch.float64, device=gu.dev())
    d_g = torch.empty(ncp, dtype=torch.float64, device=gu.dev())
    wb_g = torch.empty(ncp, dtype=torch.float64, device=gu.dev())
    iim.iim_total_pressure_problem(geo, gu.T(w.ravel()), gu.T(ux.ravel()), gu.T(uy.ravel()), None, Uinf, nu, f_g, d_g,
                                   omega_b_out=wb_g)
    assert np.abs(wb_g.cpu().numpy() - wb).max() < 1e-11 * np.abs(wb).max()
    assert np.abs(f_g.cpu().numpy().reshape(n - 1, n - 1) - f).max() < 1e-11 * np.abs(f).max()
    assert np.abs(d_g.cpu().numpy() - data).max() < 1e-11 * np.abs(data).max()
    # the wall values of an arbitrary field
    field = np.where((P.phi >= 0)[1:-1, 1:-1], inputs.vortex_field(P.grid, 5, count=9, sigma=0.3)[1:-1, 1:-1], 0.0)
    hw = torch.empty(ncp, dtype=torch.float64, device=gu.dev())
    iim.iim_wall_values(geo, gu.T(field.ravel()), hw)
    ref = pr.wall_values(S, field)
    assert np.abs(hw.cpu().numpy() - ref).max() < 1e-13 * np.abs(ref).max()
    geo.close()


@pytest.mark.parametrize("mode", ["fp64", "mixed_precond"])
def test_total_pressure_matches_oracle(mode):
    """The whole global method (right-hand side, wall datum, Neumann solve, surface values) against
    the oracle's, element by element."""
    n = 128
    P, S, w, ux, uy, Uinf = _flow_snapshot(n)
    T = tr.TransportSetup(S)
    nu = 0.004
    SN = op.Setup(P, wall="neumann", wall_data=np.zeros(S.geo["cp"]["t"].size))
    H_ref, Hw_ref, _, _, _, _ = pr.total_pressure(T, SN, w, ux, uy, Uinf, nu)
    geo = _neumann_geometry(P)
    NXY = (n - 1) ** 2
    H = torch.empty(NXY, dtype=torch.float64, device=gu.dev())
    Hw = torch.empty(geo.n_control, dtype=torch.float64, device=gu.dev())
    prec, pc, rtol, tol = ((iim.IIM_FP64, 0, 1e-12, 1e-10) if mode == "fp64" else (iim.IIM_MIXED, 1, 1e-10, 1e-8))
    st = iim.iim_total_pressure(geo, gu.T(w.ravel()), gu.T(ux.ravel()), gu.T(uy.ravel()), Uinf, nu, H, H_wall_out=Hw,
                                opts=iim.default_opts(prec=prec, rtol=rtol, precond=pc, restart=64, max_iter=3000))
    scale = np.abs(H_ref).max()
    assert np.abs(H.cpu().numpy().reshape(n - 1, n - 1) - H_ref[1:-1, 1:-1]).max() < tol * scale, st
    assert np.abs(Hw.cpu().numpy() - Hw_ref).max() < tol * scale
    geo.close()


def test_total_pressure_needs_neumann_geometry():
    P, S, w, ux, uy, Uinf = _flow_snapshot(64)
    geo = gu.setup(P)
    H = torch.empty(63 * 63, dtype=torch.float64, device=gu.dev())
    with pytest.raises(iim.IIMError):
        iim.iim_total_pressure(geo, gu.T(w.ravel()), gu.T(ux.ravel()), gu.T(uy.ravel()), Uinf, 0.004, H)
    geo.close()


def test_total_pressure_full_size_cylinder_flow_residual():
    """At the 1024 x 512 flow-past-a-cylinder size: the mixed, preconditioned total-pressure solve
    reaches the 1e-10 un-reduced residual of the oracle's Neumann system (evaluated by the oracle
    on the GPU's H, right-hand side and wall datum), and the datum and right-hand side match the
    oracle's at sampled control points and nodes."""
    P0 = inputs.c2_cylinder_flow(1024, 512)
    g = P0.grid
    P = inputs.Problem(grid=g, phi=P0.phi, regions=P0.regions, modes=[0], omega=P0.omega, psi_box=np.zeros(2 * (g.nx + g.ny)),
                       psi_b_fn=lambda x, y, k: np.zeros_like(x), psibar=np.zeros(1), gamma=None, exact=None)
    X, Y = g.nodes()
    fl = (P.phi >= 0)[1:-1, 1:-1]
    # a wake-like vorticity behind the cylinder and the velocity of a free stream plus that field
    w = np.where(fl, inputs.vortex_field(g, 3, count=40, sigma=0.12, lo=(-0.5, -1.0), hi=(4.0, 1.0))[1:-1, 1:-1], 0.0)
    geo_flow = gu.setup(inputs.Problem(grid=g, phi=P.phi, regions=P.regions, modes=[0], omega=w, psi_box=P0.psi_box,
                                       psi_b_fn=lambda x, y, k: np.zeros_like(x), psibar=np.zeros(1), gamma=None,
                                       exact=None))
    NXY = (g.nx - 1) * (g.ny - 1)
    psi = torch.empty(NXY, dtype=torch.float64, device=gu.dev())
    ux, uy = torch.empty_like(psi), torch.empty_like(psi)
    ncp = geo_flow.n_control
    iim.iim_poisson_solve(geo_flow, gu.T(w.ravel()), torch.zeros(ncp, dtype=torch.float64, device=gu.dev()),
                          gu.T(P0.psi_box), None, torch.zeros(1, dtype=torch.float64, device=gu.dev()), psi, ux, uy,
                          opts=iim.default_opts(prec=iim.IIM_MIXED, rtol=1e-10))
    geo_flow.close()
    geo = _neumann_geometry(P)
    nu = 0.005
    f_g = torch.empty(NXY, dtype=torch.float64, device=gu.dev())
    d_g = torch.empty(ncp, dtype=torch.float64, device=gu.dev())
    iim.iim_total_pressure_problem(geo, gu.T(w.ravel()), ux, uy, None, (1.0, 0.0), nu, f_g, d_g)
    H = torch.empty(NXY, dtype=torch.float64, device=gu.dev())
    st = iim.iim_total_pressure(geo, gu.T(w.ravel()), ux, uy, (1.0, 0.0), nu, H,
                                opts=iim.default_opts(prec=iim.IIM_MIXED, rtol=1e-10, precond=1))
    assert st["rel_res"] <= 1e-10
    f, data = f_g.cpu().numpy(), d_g.cpu().numpy()
    SN = op.Setup(P, wall="neumann", wall_data=data)
    Hn = np.zeros((g.ny + 1, g.nx + 1))
    Hn[1:-1, 1:-1] = H.cpu().numpy().reshape(g.ny - 1, g.nx - 1)
    assert op.residual(SN, Hn, np.zeros(1), omega=f.reshape(g.ny - 1, g.nx - 1), ring=np.zeros(2 * (g.nx + g.ny))) <= 1e-10
    # sampled rows of the right-hand side against the oracle's centred differences (the rows
    # away from the body need no extension: plain products of the given fields)
    uxn, uyn = ux.cpu().numpy().reshape(g.ny - 1, g.nx - 1), uy.cpu().numpy().reshape(g.ny - 1, g.nx - 1)
    fr = f.reshape(g.ny - 1, g.nx - 1)
    h = g.h
    for j in (40, 200, 400):
        for i in (700, 800, 900):
            q = lambda a, b: uyn[b, a] * w[b, a]
            r = lambda a, b: uxn[b, a] * w[b, a]
            ref = -((q(i + 1, j) - q(i - 1, j)) - (r(i, j + 1) - r(i, j - 1))) / (2 * h)
            assert abs(fr[j, i] - ref) <= 1e-12 * max(1.0, abs(ref))
    geo.close()
