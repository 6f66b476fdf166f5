"""Pins of the oracle's transport step (Sec. 3, 5.1, 5.3, 5.5, App. B)."""
import math
import os

import numpy as np
import pytest

from oracle import poisson as op
from oracle import transport as tr
from paper_2109_13628_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rk3_stability_polygon.txt")


def body_problem(n, half=2.0, seed=0):
    g = inputs.square_grid(n, half)
    X, Y = g.nodes()
    a = inputs.phi_circle(X, Y, -0.8, -0.7, 0.45)
    b = inputs.phi_star(X, Y, 0.7, 0.6, 0.45, 0.08, 4)
    phi = inputs.union(a, b)
    regions = [inputs.region_around(g, a), inputs.region_around(g, b)]
    return inputs.Problem(grid=g, phi=phi, regions=regions, modes=[1, 1], omega=np.zeros((n - 1, n - 1)),
                          psi_box=np.zeros(4 * n), psi_b_fn=lambda x, y, k: np.zeros_like(x), psibar=np.zeros(2),
                          gamma=None, exact=None)


def test_rk3_polygon_golden_and_dt_formula():
    pts = np.loadtxt(GOLDEN)
    assert pts.shape == (3, 2)
    assert tr.STAB_C == pts[1, 0] and tr.STAB_R == pts[2, 1]
    h, nu = 0.01, 0.003
    # pure diffusion and pure advection end points of the polygon edge
    assert math.isclose(tr.dt_max(np.zeros(3), np.zeros(3), nu, h), pts[2, 1] * h * h / nu)
    assert math.isclose(tr.dt_max(np.array([2.0]), np.array([-1.0]), 1e-300, h), pts[1, 0] * h / 3.0, rel_tol=1e-12)
    # the (C, r) point of dt_max lies on the segment between the two vertices
    dt = tr.dt_max(np.array([0.7]), np.array([0.2]), nu, h)
    C, r = 0.9 * dt / h, nu * dt / h / h
    assert abs(C / pts[1, 0] + r / pts[2, 1] - 1.0) < 1e-12


def test_williamson_rk3_stability_polynomial():
    """Any 3-stage third-order RK has R(z) = 1 + z + z^2/2 + z^3/6 (closed form)."""
    for z in (-0.3, 0.1 + 0.5j, -1.2 - 0.7j):
        q, dq = 1.0 + 0j, 0.0 + 0j
        for s in range(3):
            dq = tr.RK3_A[s] * dq + z * q
            q = q + tr.RK3_B[s] * dq
        assert abs(q - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-14


@pytest.mark.parametrize("n", [64, 96])
def test_transport_rhs_exact_for_bilinear_vorticity(n):
    """omega bilinear, u linear and divergence free: every stencil and extension is exact, so
    d omega/dt = -u . grad omega exactly, also next to the bodies (away from the box)."""
    P = body_problem(n)
    S = op.Setup(P)
    T = tr.TransportSetup(S)
    Xi, Yi = P.grid.interior()
    a, b, c, d = 0.7, -0.4, 0.3, 0.9
    al, be, ga, de = 0.2, 1.1, -0.6, 0.5
    ux, uy = a + b * Yi, c + d * Xi
    w = al + be * Xi + ga * Yi + de * Xi * Yi
    cps = S.geo["cp"]
    u_b = (a + b * cps["y"], c + d * cps["x"])
    wb = al + be * cps["x"] + ga * cps["y"] + de * cps["x"] * cps["y"]
    rhs, Fx, Fy, _ = tr.transport_rhs(T, w, ux, uy, u_b, (0.0, 0.0), 0.01, omega_b=wb)
    exact = -(ux * (be + de * Yi) + uy * (ga + de * Xi))
    fl = (P.phi >= 0)[1:-1, 1:-1]
    keep = np.zeros_like(fl)
    keep[3:-3, 3:-3] = True
    m = fl & keep
    assert np.abs(rhs - exact)[m].max() < 1e-10 * np.abs(exact).max()


@pytest.mark.parametrize("n", [64, 128])
def test_vorticity_bc_exact_for_quadratic_velocity(n):
    """Sec. 5.3 (reading): third-order velocity extension and quadratic stencils make omega_b
    exact for any quadratic velocity field."""
    P = body_problem(n)
    S = op.Setup(P)
    T = tr.TransportSetup(S)
    rng = np.random.default_rng(n)
    cx, cy = rng.normal(size=6), rng.normal(size=6)

    def quad(c, x, y):
        return c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y

    Xi, Yi = P.grid.interior()
    fl = (P.phi >= 0)[1:-1, 1:-1]
    ux, uy = np.where(fl, quad(cx, Xi, Yi), 0), np.where(fl, quad(cy, Xi, Yi), 0)
    cps = S.geo["cp"]
    x, y = cps["x"], cps["y"]
    u_b = (quad(cx, x, y), quad(cy, x, y))
    uxb, uyb = tr.extended_velocity(T, ux, uy, u_b, (0.0, 0.0))
    wb = tr.vorticity_bc(T, uxb, uyb, u_b)
    # omega = d(uy)/dx - d(ux)/dy
    exact = (cy[1] + 2 * cy[3] * x + cy[4] * y) - (cx[2] + cx[4] * x + 2 * cx[5] * y)
    assert np.abs(wb - exact).max() < 1e-8 * (1 + np.abs(exact).max())


def test_telescoping_conservation_and_kelvin():
    """Eq. 2dintconserve: h^2 sum_R d omega/dt = -h sum_dR (f+q).n on fluid regions, exactly."""
    P = body_problem(96)
    S = op.Setup(P)
    T = tr.TransportSetup(S)
    g = P.grid
    w = inputs.vortex_field(g, 3, count=10, sigma=0.3)[1:-1, 1:-1]
    fl = (P.phi >= 0)[1:-1, 1:-1]
    w = np.where(fl, w, 0)
    psi, pb = op.solve_unreduced(S, omega=w, gamma=op.gamma_from_regions(P))
    ux, uy = op.velocity(S, psi, pb)
    cps = S.geo["cp"]
    zero = (np.zeros(len(cps["t"])), np.zeros(len(cps["t"])))
    rhs, Fx, Fy, _ = tr.transport_rhs(T, w, ux, uy, zero, (0.0, 0.0), 0.01)
    h = g.h
    for region in [(10, 20, 60, 80), (70, 90, 5, 12), (40, 41, 85, 86)]:
        lx, rx, ly, ry = region
        assert fl[ly - 1:ry, lx - 1:rx].all()
        lhs = h * h * rhs[ly - 1:ry, lx - 1:rx].sum()
        assert abs(lhs + tr.region_flux(S, Fx, Fy, region)) < 1e-12 * (np.abs(rhs).max() * h * h * 400 + 1e-300)
    dG = tr.kelvin_rhs(S, Fx, Fy)
    assert np.all(np.isfinite(dG))


def test_rk3_step_conserves_total_circulation():
    """Discrete Kelvin (Sec. 5.1): sum_k Gamma_k + h^2 (sum of omega outside every R_k) is
    constant over a step (vorticity far from the box, so no flux leaves the box): the Kelvin
    ODE takes exactly the flux that leaves each R_k."""
    P = body_problem(64)
    S = op.Setup(P)
    T = tr.TransportSetup(S)
    g = P.grid
    X, Y = g.nodes()
    w = inputs.gaussian_vortices(X, Y, [(0.4, -0.6), (-0.6, 0.7)], [1.0, -0.7], 0.12)[1:-1, 1:-1]
    fl = (P.phi >= 0)[1:-1, 1:-1]
    w = np.where(fl, w, 0)
    gam = op.gamma_from_regions(P) + np.array([0.02, -0.03])
    ncp = S.geo["cp"]["t"].size
    u_b = (np.zeros(ncp), np.zeros(ncp))
    h = g.h

    def total(wv, gv):
        inside = np.zeros_like(fl)
        for (lx, rx, ly, ry) in P.regions:
            inside[ly - 1:ry, lx - 1:rx] = True
        return gv.sum() + h * h * wv[~inside].sum()

    w1, g1, dt, pb = tr.rk3_step(T, w, gam, u_b, (0.0, 0.0), 0.01, 0.5)
    assert dt > 0
    assert abs(total(w1, g1) - total(w, gam)) < 1e-12
    assert abs(g1 - gam).max() > 1e-6      # the bodies did exchange circulation
    assert np.abs(w1[~fl]).max() == 0.0


def test_rk3_third_order_in_time():
    """Temporal refinement at fixed h (Sec. 5.5, smooth advection-dominated case): a weak
    Gaussian vortex carried by the free stream (1, 0.3) through an empty box, the full step
    (velocity reconstruction, transport, Williamson RK3) integrated to t = 0.08 with dt = 0.04,
    0.02, 0.01 against dt = 0.005; the error falls by about 2^3 per halving.  (With bodies the
    upwind selection switches where the face velocity changes sign, which is not smooth in time.)"""
    n = 64
    g = inputs.square_grid(n)
    X, Y = g.nodes()
    P = inputs.Problem(grid=g, phi=np.ones_like(X), regions=[], modes=[], omega=np.zeros((n - 1, n - 1)),
                       psi_box=inputs.box_ring(g, 1.0 * Y - 0.3 * X), psi_b_fn=lambda x, y, k: np.zeros_like(x),
                       psibar=np.zeros(0), gamma=None, exact=None)
    S = op.Setup(P)
    T = tr.TransportSetup(S)
    w0 = (0.05 * inputs.gaussian_vortices(X, Y, [(-0.5, -0.2)], [1.0], 0.3))[1:-1, 1:-1]
    u_b = (np.zeros(0), np.zeros(0))

    def run(dt, steps):
        w, gm = w0.copy(), np.zeros(0)
        for _ in range(steps):
            w, gm, _, _ = tr.rk3_step(T, w, gm, u_b, (1.0, 0.3), 0.002, 0.5, dt=dt, psibar=np.zeros(0))
        return w

    ref = run(0.005, 16)
    errs = [np.abs(run(dt, steps) - ref).max() for dt, steps in ((0.04, 2), (0.02, 4), (0.01, 8))]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 2.6, (errs, orders)


def test_rk3_stage_times_integrate_quadratics_exactly():
    """The stage times c = (0, 1/3, 3/4) belong to the Williamson coefficients (Sec. 5.5): the
    2N-storage update of y' = p(t), with p read at t + c_s dt, integrates every polynomial of
    degree <= 2 exactly (third order) and misses t^3, and each stage's state is y at its stage
    time for linear p (so a wall velocity linear in time is seen at the right time).  A wrong c
    or a wrong A/B pairing breaks one of these."""
    def integrate(p, t, dt):
        y, dy, states = 0.0, 0.0, []
        for s in range(3):
            states.append(y)
            dy = tr.RK3_A[s] * dy + dt * p(t + tr.RK3_C[s] * dt)
            y += tr.RK3_B[s] * dy
        return y, states

    t, dt = 0.3, 0.7
    for k in range(3):
        y, _ = integrate(lambda x: (k + 1) * x ** k, t, dt)
        assert abs(y - ((t + dt) ** (k + 1) - t ** (k + 1))) < 1e-14
    y3, _ = integrate(lambda x: 4 * x ** 3, t, dt)
    assert abs(y3 - ((t + dt) ** 4 - t ** 4)) > 1e-3
    _, states = integrate(lambda x: 1.0, t, dt)
    assert np.allclose(states, [c * dt for c in tr.RK3_C], atol=1e-15)


def test_vorticity_bc_second_order_with_exact_velocity():
    """Sec. 5.3 stencils (the reading of the missing figure used here): fed the exact Lamb-Oseen
    velocity around the Sec. 6.1 cylinder (extended into the body with u_b as the transport
    step does), the wall vorticity converges at second order at every control point."""
    c = inputs.LAMB_OSEEN_CYLINDER
    errs = []
    for n in (128, 256):
        P = inputs.lamb_oseen_cylinder(n)
        S = op.Setup(P)
        T = tr.TransportSetup(S)
        cp = S.geo["cp"]
        X, Y = P.grid.nodes()
        _, ux, uy = inputs.lamb_oseen(X, Y, c["xc"], c["yc"], c["gamma"], c["nu"] * c["t0"])
        wex, bx, by = inputs.lamb_oseen(cp["x"], cp["y"], c["xc"], c["yc"], c["gamma"], c["nu"] * c["t0"])
        uxb, uyb = tr.extended_velocity(T, ux[1:-1, 1:-1], uy[1:-1, 1:-1], (bx, by), (0.0, 0.0))
        wb = tr.vorticity_bc(T, uxb, uyb, (bx, by))
        errs.append(np.abs(wb - wex).max())
    assert math.log2(errs[0] / errs[1]) > 1.8, errs
    assert errs[1] < 0.1 * np.abs(wex).max(), errs
