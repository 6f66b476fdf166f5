"""Pins of the oracle's total-pressure problem (Sec. 5.4) and of the Neumann variant of the
extrapolation (Sec. 2.1) against what the mathematics fixes: polynomial reproduction, exactness
of the discrete solve for bicubic fields, second-order convergence on a smooth field, exactness
of the right-hand side, wall-datum and surface-value stencils on low-degree fields, and the
right-hand side of an exact Navier-Stokes flow (circular Couette flow around a stationary
cylinder)."""
import numpy as np
import pytest

from oracle import extrapolation as ex
from oracle import poisson as op
from oracle import pressure as pr
from oracle import transport as tr
from paper_2109_13628_gb300 import inputs


def _neumann_data(S, grad_fn):
    """d . grad f at every control point, d the grid direction from the solid node to the fluid."""
    cps = S.geo["cp"]
    gx, gy = grad_fn(cps["x"], cps["y"])
    return (cps["fi"] - cps["si"]) * gx + (cps["fj"] - cps["sj"]) * gy


def _bicubic_grad(x, y, c):
    gx, gy = np.zeros_like(x), np.zeros_like(x)
    for a in range(4):
        for b in range(4):
            if a:
                gx = gx + c[a, b] * a * x ** (a - 1) * y ** b
            if b:
                gy = gy + c[a, b] * b * x ** a * y ** (b - 1)
    return gx, gy


def test_hermite_weights_reproduce_cubics():
    rng = np.random.default_rng(3)
    for _ in range(20):
        a = rng.uniform(0.0, 1.0)
        c = rng.normal(size=4)
        p = np.polynomial.Polynomial(c)
        w = ex.hermite_weights(a)
        got = w[0] * p.deriv()(a) + sum(w[k] * p(m) for k, m in ((1, 2.0), (2, 3.0), (3, 4.0)))
        assert abs(got - p(0.0)) <= 1e-12 * (1 + np.abs(c).sum())


@pytest.mark.parametrize("n", [64, 128])
def test_neumann_solve_exact_for_bicubic_fields(n):
    """With the cubic Neumann extrapolation and the five-point Laplacian both exact on fields of
    degree <= 3 in each variable, the discrete solution is the field itself, around a circle, an
    ellipse and a nonconvex star, in the un-reduced form and in the Schur-complement form."""
    P = inputs.bicubic_bodies(n, seed=1, circulation=False)
    c = inputs.bicubic_coeffs(1)
    S0 = op.Setup(P, wall="neumann", wall_data=np.zeros(1))
    S = op.Setup(P, wall="neumann", wall_data=_neumann_data(S0, lambda x, y: _bicubic_grad(x, y, c)))
    fl = ~S.solid
    scale = np.abs(P.exact).max()
    psi, _ = op.solve_unreduced(S, psibar=np.zeros(3))
    assert np.abs(np.where(fl, psi - P.exact, 0.0)).max() < 1e-11 * scale
    psi2, _, it, rel = op.solve_schur(S, psibar=np.zeros(3), tol=1e-13)
    assert rel < 1e-12
    assert np.abs(np.where(fl, psi2 - P.exact, 0.0)).max() < 1e-10 * scale
    assert op.residual(S, psi2, np.zeros(3)) < 1e-11


def test_neumann_rejects_circulation_bodies():
    P = inputs.bicubic_bodies(64, seed=1, circulation=True)
    with pytest.raises(ValueError):
        op.Setup(P, wall="neumann")


def test_neumann_solve_second_order_on_smooth_field():
    def H(x, y):
        return np.sin(1.3 * x + 0.4) * np.cos(0.9 * y)

    def grad(x, y):
        return 1.3 * np.cos(1.3 * x + 0.4) * np.cos(0.9 * y), -0.9 * np.sin(1.3 * x + 0.4) * np.sin(0.9 * y)

    errs = []
    for n in (48, 96, 192):
        P = inputs.c1_cylinder(n)
        X, Y = P.grid.nodes()
        ex_ = H(X, Y)
        P.omega = np.ascontiguousarray(np.where(P.phi >= 0, 2.5 * ex_, 0.0)[1:-1, 1:-1])   # -lap H = (1.69 + 0.81) H
        P.psi_box = inputs.box_ring(P.grid, ex_)
        S0 = op.Setup(P, wall="neumann", wall_data=np.zeros(1))
        S = op.Setup(P, wall="neumann", wall_data=_neumann_data(S0, grad))
        psi, _, _, _ = op.solve_schur(S, psibar=np.zeros(1), tol=1e-13)
        errs.append(np.abs(np.where(~S.solid, psi - ex_, 0.0)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 1.85, (errs, orders)


def _transport_setup(P):
    return tr.TransportSetup(op.Setup(P))


def test_rhs_exact_for_linear_velocity_and_vorticity():
    """Linear u and omega make the products quadratic: centred differences and the third-order
    extensions (fed the exact wall values) are exact, so f = -(d_x(u_y w) - d_y(u_x w)) to
    rounding at every fluid node whose stencil stays off the box."""
    P = inputs.bicubic_bodies(64, seed=2, circulation=False)
    T = _transport_setup(P)
    S = T.S
    X, Y = P.grid.nodes()
    a = np.array([0.3, -0.7, 0.4, 0.2, 0.5, -0.6, 1.1, -0.4, 0.9])
    ux = a[0] + a[1] * X + a[2] * Y
    uy = a[3] + a[4] * X + a[5] * Y
    w = a[6] + a[7] * X + a[8] * Y
    exact = -((a[4] * w + uy * a[7]) - (a[2] * w + ux * a[8]))
    cps = S.geo["cp"]
    u_b = (a[0] + a[1] * cps["x"] + a[2] * cps["y"], a[3] + a[4] * cps["x"] + a[5] * cps["y"])
    wb = a[6] + a[7] * cps["x"] + a[8] * cps["y"]
    fl = P.phi[1:-1, 1:-1] >= 0
    f, _ = pr.pressure_rhs(T, np.where(fl, w[1:-1, 1:-1], 0.0), np.where(fl, ux[1:-1, 1:-1], 0.0),
                           np.where(fl, uy[1:-1, 1:-1], 0.0), u_b, (0.0, 0.0), omega_b=wb)
    inner = np.zeros_like(fl)
    inner[1:-1, 1:-1] = True
    m = fl & inner
    err = np.abs(np.where(m, f - exact[1:-1, 1:-1], 0.0)).max()
    assert err < 1e-11, err


def _couette(P, A=1.0, R=0.5):
    """Circular Couette flow outside a stationary cylinder of radius R at the origin:
    u_theta = A (r - R^2 / r), omega = 2 A, -div(u x omega k) = -omega^2 = -4 A^2."""
    X, Y = P.grid.nodes()
    r2 = np.maximum(X * X + Y * Y, 1e-300)     # the origin is inside the cylinder (masked)
    ux = -A * (Y - R * R * Y / r2)
    uy = A * (X - R * R * X / r2)
    fl = P.phi[1:-1, 1:-1] >= 0
    return (np.where(fl, 2.0 * A, 0.0), np.where(fl, ux[1:-1, 1:-1], 0.0), np.where(fl, uy[1:-1, 1:-1], 0.0))


def test_rhs_second_order_on_couette_flow():
    """Max-norm error of f next to the wall, with omega_b from the vorticity boundary condition:
    second order (the per-refinement order wanders with where the crossings fall)."""
    errs = []
    for n in (64, 128, 256):
        P = inputs.c1_cylinder(n)
        T = _transport_setup(P)
        ncp = len(T.S.geo["cp"]["t"])
        w, ux, uy = _couette(P)
        f, wb = pr.pressure_rhs(T, w, ux, uy, (np.zeros(ncp), np.zeros(ncp)), (0.0, 0.0))
        fl = P.phi[1:-1, 1:-1] >= 0
        inner = np.zeros_like(fl)
        inner[1:-1, 1:-1] = True
        errs.append(np.abs(np.where(fl & inner, f + 4.0, 0.0)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 1.6 and np.log2(errs[0] / errs[-1]) / 2 > 1.75, (errs, orders)


def test_wall_data_exact_for_biquadratic_vorticity():
    """The cross-line stencil is exact for omega of degree <= 2 in each variable, so the datum is
    nu d . (-d_y omega, d_x omega) to rounding wherever a two-row stencil exists."""
    P = inputs.bicubic_bodies(96, seed=4, circulation=False)
    T = _transport_setup(P)
    S = T.S
    X, Y = P.grid.nodes()
    c = np.random.default_rng(5).normal(size=(3, 3))

    def om(x, y):
        return sum(c[a, b] * x ** a * y ** b for a in range(3) for b in range(3))

    def om_grad(x, y):
        gx = sum(c[a, b] * a * x ** (a - 1) * y ** b for a in range(1, 3) for b in range(3))
        gy = sum(c[a, b] * b * x ** a * y ** (b - 1) for a in range(3) for b in range(1, 3))
        return gx, gy

    nu = 0.01
    cps = S.geo["cp"]
    fl = P.phi[1:-1, 1:-1] >= 0
    got = pr.wall_data(T, np.where(fl, om(X, Y)[1:-1, 1:-1], 0.0), om(cps["x"], cps["y"]), nu)
    gx, gy = om_grad(cps["x"], cps["y"])
    exact = _neumann_data(S, lambda x, y: (-nu * gy, nu * gx))
    err = np.abs(got - exact)
    assert np.median(err) < 1e-12
    # the nonconvex star leaves a few control points with a one-row (first-order) stencil only
    assert (err > 1e-10).mean() < 0.02


def test_wall_values_exact_for_quadratic_fields():
    P = inputs.c1_cylinder(64)
    S = op.Setup(P)
    X, Y = P.grid.nodes()
    F = 0.4 + 0.3 * X - 0.8 * Y + 0.5 * X * X - 0.2 * X * Y + 0.7 * Y * Y + 0.3 * X * X * Y * Y
    cps = S.geo["cp"]
    got = pr.wall_values(S, np.where(P.phi >= 0, F, 0.0)[1:-1, 1:-1])
    ex_ = 0.4 + 0.3 * cps["x"] - 0.8 * cps["y"] + 0.5 * cps["x"] ** 2 - 0.2 * cps["x"] * cps["y"] + \
        0.7 * cps["y"] ** 2 + 0.3 * cps["x"] ** 2 * cps["y"] ** 2
    assert np.abs(got - ex_).max() < 1e-12


def test_total_pressure_couette_flow():
    """The global method on circular Couette flow around the stationary cylinder, with the exact
    total pressure H = A^2 (r^2 - 2 R^2 ln r) + const on the box.  omega is constant, so the wall
    datum is only the derivative of the vorticity boundary condition's error, and H is one
    constant on the wall.
      * With the exact right-hand side -4 A^2 (the Neumann solve, wall datum and surface values):
        H converges to the exact field, faster than first order.
      * With the right-hand side computed from the flow: the box layer, where the flow solver's
        box values (u = U_inf, omega = 0) stand for the Couette field's, adds a first-order term;
        the surface values stay one constant to the accuracy of the datum."""
    A, R = 1.0, 0.5
    err_exact_f, err_full, spread = [], [], []
    for n in (32, 64, 128):
        P = inputs.c1_cylinder(n)
        X, Y = P.grid.nodes()
        r2 = np.maximum(X * X + Y * Y, 1e-300)
        Hex = A * A * (r2 - R * R * np.log(r2))
        ring = inputs.box_ring(P.grid, Hex)
        T = _transport_setup(P)
        SN = op.Setup(P, wall="neumann", wall_data=np.zeros(len(T.S.geo["cp"]["t"])))
        w, ux, uy = _couette(P)
        H, Hw, f, data, wb, it = pr.total_pressure(T, SN, w, ux, uy, (0.0, 0.0), 0.01, H_box=ring)
        err_full.append(np.abs(np.where(~SN.solid, H - Hex, 0.0)).max())
        spread.append(np.ptp(Hw))
        fe = np.where(P.phi[1:-1, 1:-1] >= 0, -4.0 * A * A, 0.0)
        H2, _, _, _ = op.solve_schur(SN, omega=fe, ring=ring, psibar=np.zeros(1), tol=1e-13)
        err_exact_f.append(np.abs(np.where(~SN.solid, H2 - Hex, 0.0)).max())
    assert np.log2(err_exact_f[0] / err_exact_f[2]) / 2 > 1.1, err_exact_f
    assert err_exact_f[2] < 5e-4, err_exact_f
    assert all(err_full[k + 1] < 0.6 * err_full[k] for k in range(2)), err_full
    assert spread[2] < spread[0] / 4.0 and spread[2] < 5e-4, spread
