"""Pins of the oracle's Poisson path against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form (eigenvectors of
the five-point Laplacian, polynomial exactness of the IIM discretization, exact circle
crossings, discrete Gauss theorem), an independent construction (sine-matrix DST, the
un-reduced system against the Schur form), or a convergence order stated by the paper.
"""
import math

import numpy as np
import pytest

from oracle import extrapolation as ex
from oracle import geometry as geom
from oracle import poisson as op
from paper_2109_13628_gb300 import inputs


# ----------------------------------------------------------------------------- DST / box solver
@pytest.mark.parametrize("N", [1, 7, 15, 31, 63])
def test_dst1_fft_matches_sine_matrix(N):
    x = np.random.default_rng(N).normal(size=(3, N))
    assert np.allclose(op.dst1(x), op.dst1_matrix(x), rtol=0, atol=1e-12 * N)


def test_dst1_is_its_own_inverse_up_to_n_over_2():
    x = np.random.default_rng(1).normal(size=31)
    assert np.allclose(op.dst1(op.dst1(x)) * 2.0 / 32, x, atol=1e-13)


@pytest.mark.parametrize("nx,ny", [(16, 16), (32, 16), (64, 128)])
def test_sine_modes_are_eigenvectors(nx, ny):
    """-nabla_h^2 sin(k pi x~) sin(l pi y~) = (lam_k + mu_l) sin sin (closed form)."""
    h = 1.0 / 8
    i = np.arange(0, nx + 1)
    j = np.arange(0, ny + 1)
    for k, l in ((1, 1), (3, 2), (nx - 1, ny - 1)):
        mode = np.outer(np.sin(np.pi * l * j / ny), np.sin(np.pi * k * i / nx))
        lam = 4.0 * math.sin(math.pi * k / (2 * nx)) ** 2 / h**2 + 4.0 * math.sin(math.pi * l / (2 * ny)) ** 2 / h**2
        assert np.allclose(op.neg_laplacian_5pt(mode, h), lam * mode[1:-1, 1:-1], atol=1e-9 * lam)
        u = op.poisson_box(lam * mode[1:-1, 1:-1], h)
        assert np.allclose(u, mode[1:-1, 1:-1], atol=1e-12)


def test_box_solver_inverts_laplacian_with_box_data():
    rng = np.random.default_rng(3)
    nx, ny, h = 32, 16, 0.1
    u = rng.normal(size=(ny + 1, nx + 1))
    g = inputs.Grid(0, nx * h, 0, ny * h, nx, ny)
    ring = inputs.box_ring(g, u)
    f = op.neg_laplacian_5pt(u, h)
    assert np.allclose(op.poisson_box(f, h, ring), u[1:-1, 1:-1], atol=1e-11)


# ----------------------------------------------------------------------------- geometry
def test_circle_crossings_fourth_order():
    """App. A: control points located to O(h^4) (exact crossings of a circle are known)."""
    errs = []
    for n in (32, 64, 128):
        g = inputs.square_grid(n)
        X, Y = g.nodes()
        R = 0.7
        phi = inputs.phi_circle(X, Y, 0.1, -0.05, R)
        cp = geom.control_points(g, phi)
        r = np.hypot(cp["x"] - 0.1, cp["y"] + 0.05)
        errs.append(np.abs(r - R).max())
        assert len(cp["t"]) > 0 and (cp["t"] >= 0).all() and (cp["t"] <= 1).all()
    assert errs[0] / errs[1] > 12 and errs[1] / errs[2] > 12, errs


def test_crossings_lie_between_solid_and_fluid_nodes():
    g = inputs.square_grid(64)
    X, Y = g.nodes()
    phi = inputs.phi_star(X, Y, 0.0, 0.0, 0.8, 0.2, 5)
    cp = geom.control_points(g, phi)
    assert (phi[cp["sj"], cp["si"]] < 0).all() and (phi[cp["fj"], cp["fi"]] >= 0).all()
    assert (np.abs(cp["si"] - cp["fi"]) + np.abs(cp["sj"] - cp["fj"]) == 1).all()
    # every sign change of phi along a grid line gives exactly one control point
    s = phi < 0
    n_expected = int((s[:, 1:] != s[:, :-1]).sum() + (s[1:, :] != s[:-1, :]).sum())
    assert len(cp["t"]) == n_expected


def test_affected_sets_by_definition_on_tiny_case():
    phi = np.ones((6, 6))
    phi[2, 2] = phi[2, 3] = -1.0
    plus, minus = geom.affected_points(phi)
    assert set(zip(*np.nonzero(minus))) == {(2, 2), (2, 3)}
    assert set(zip(*np.nonzero(plus))) == {(1, 2), (1, 3), (3, 2), (3, 3), (2, 1), (2, 4)}


# ----------------------------------------------------------------------------- extrapolation
@pytest.mark.parametrize("degree,with_bc", [(3, True), (2, True), (2, False)])
def test_ghosts_reproduce_polynomials(degree, with_bc):
    """Sec. 2.1: the extrapolation is exact for polynomials of degree <= n along grid lines,
    hence for p(x, y) with degree <= n in each variable, for every usable direction."""
    g = inputs.square_grid(64)
    X, Y = g.nodes()
    phi = inputs.union(inputs.phi_circle(X, Y, -0.9, 0.0, 0.45), inputs.phi_star(X, Y, 0.8, 0.2, 0.55, 0.1, 4))
    geo = geom.process_geometry(g, phi, [inputs.region_around(g, inputs.phi_circle(X, Y, -0.9, 0.0, 0.45)),
                                         inputs.region_around(g, inputs.phi_star(X, Y, 0.8, 0.2, 0.55, 0.1, 4))])
    c = np.random.default_rng(5).normal(size=(4, 4))
    c[degree + 1:, :] = 0
    c[:, degree + 1:] = 0
    p = inputs.bicubic(X, Y, c)
    nodes, Gpsi, Gbc, nval = ex.ghost_operator(geo, phi, degree=degree, with_bc=with_bc)
    bc = inputs.bicubic(geo["cp"]["x"], geo["cp"]["y"], c)
    ext = ex.extend(p, phi, (nodes, Gpsi, Gbc, nval), bc if with_bc else None)
    for (i, j) in nodes:
        assert abs(ext[j, i] - p[j, i]) < 1e-10 * (1 + abs(p).max())
    assert (nval >= 1).all() and (nval <= 4).all()


def test_lagrange_weights_partition_unity_and_cancel_at_boundary():
    for t in (0.0, 1e-9, 0.3, 1.0):
        w = ex.lagrange_at([1 - t, 2, 3, 4], 0.0)
        assert abs(w.sum() - 1) < 1e-14
    # crossing exactly on the ghost node: the ghost equals the boundary value
    assert np.allclose(ex.lagrange_at([0.0, 2, 3, 4], 0.0), [1, 0, 0, 0])


# ----------------------------------------------------------------------------- whole solve
@pytest.mark.parametrize("n", [48, 96])
@pytest.mark.parametrize("circulation", [True, False])
def test_polynomial_exactness_unreduced_and_schur(n, circulation):
    """A bicubic psi* makes the five-point Laplacian and every 1D extrapolation exact, so the
    discrete solution equals psi* at each fluid node and psibar_k the chosen offsets."""
    P = inputs.bicubic_bodies(n, seed=n, circulation=circulation)
    S = op.Setup(P)
    gam = np.array([op.discrete_circulation(P.exact, r) for r in P.regions])
    pb_in = None if circulation else P.psibar
    fl = P.phi >= 0
    scale = np.abs(P.exact).max()
    psi, pb = op.solve_unreduced(S, gamma=gam, psibar=pb_in)
    assert np.abs(psi - P.exact)[fl].max() < 1e-12 * scale
    assert np.allclose(pb, P.psibar, atol=1e-11)
    psi2, pb2, it, rel = op.solve_schur(S, gamma=gam, psibar=pb_in)
    assert np.abs(psi2 - P.exact)[fl].max() < 1e-12 * scale
    assert np.allclose(pb2, P.psibar, atol=1e-10)
    assert op.residual(S, psi, pb, gamma=gam) < 1e-13


def test_schur_form_matches_unreduced_on_vortex_field():
    """Non-polynomial data: the two forms of Sec. 4.2 give the same fluid psi (this decides the
    Schur sign reading); flipping the sign of A P E_a breaks the agreement."""
    P = inputs.bicubic_bodies(64, seed=1, circulation=True)
    g = P.grid
    X, Y = g.nodes()
    w = inputs.vortex_field(g, 4, count=12, sigma=0.25)
    P.omega = np.where(P.phi >= 0, w, 0.0)[1:-1, 1:-1]
    S = op.Setup(P)
    gam = op.gamma_from_regions(P)
    psi, pb = op.solve_unreduced(S, gamma=gam)
    psi2, pb2, it, rel = op.solve_schur(S, gamma=gam)
    fl = P.phi >= 0
    assert np.abs(psi - psi2)[fl].max() < 1e-11 * np.abs(psi).max()
    assert np.allclose(pb, pb2, rtol=1e-10, atol=1e-12)
    assert op.residual(S, psi2, pb2, gamma=gam) < 1e-12


def test_discrete_gauss_identity():
    """Eq. poissonintconservation: -h^2 sum_R nabla_h^2 psi = -h sum_dR (grad_h psi).n."""
    rng = np.random.default_rng(9)
    psi = rng.normal(size=(41, 37))
    h = 0.07
    region = (5, 20, 7, 30)
    lx, rx, ly, ry = region
    lap = -op.neg_laplacian_5pt(psi, h)
    lhs = -h * h * lap[ly - 1:ry, lx - 1:rx].sum()
    assert abs(lhs - op.discrete_circulation(psi, region)) < 1e-10 * np.abs(psi).sum()


def test_circulation_independent_of_region():
    """Sec. 5.1: growing R_k by one cell while adding the vorticity of the added ring to
    Gamma_k leaves psi unchanged."""
    P = inputs.bicubic_bodies(64, seed=2, circulation=True)
    g = P.grid
    w = inputs.vortex_field(g, 5, count=12, sigma=0.25)
    P.omega = np.where(P.phi >= 0, w, 0.0)[1:-1, 1:-1]
    gam = op.gamma_from_regions(P) + np.array([0.1, -0.2, 0.05])
    S = op.Setup(P)
    psi, pb = op.solve_unreduced(S, gamma=gam)
    lx, rx, ly, ry = P.regions[0]
    big = (lx - 1, rx + 1, ly - 1, ry + 1)
    gam2 = gam.copy()
    gam2[0] += g.h ** 2 * (op.region_sum(P.omega, big) - op.region_sum(P.omega, P.regions[0]))
    P.regions = [big] + list(P.regions[1:])
    S2 = op.Setup(P)
    psi2, pb2 = op.solve_unreduced(S2, gamma=gam2)
    assert np.abs(psi - psi2).max() < 1e-11 * np.abs(psi).max()
    for k, r in enumerate(P.regions):
        assert abs(op.discrete_circulation(psi2, r) - gam2[k]) < 1e-10


def test_second_order_convergence_c1():
    """Sec. 4.3 / Sec. 6.1: second-order L-infinity convergence of psi up to the boundary."""
    errs = []
    for n in (64, 128, 256):
        P = inputs.c1_cylinder(n)
        S = op.Setup(P)
        psi, pb = op.solve_unreduced(S, psibar=np.zeros(1))
        fl = P.phi >= 0
        errs.append(np.abs(psi - P.exact)[fl].max())
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 1.8, (errs, rates)


def test_velocity_second_order_lamb_oseen():
    """Sec. 4.3: velocity of a Lamb-Oseen vortex around a body converges at second order."""
    from scipy.special import exp1
    errs = []
    gamma, nu_t, x0, y0 = 1.0, 0.05, 0.35, 0.3
    for n in (64, 128, 256):
        g = inputs.square_grid(n)
        X, Y = g.nodes()
        phi = inputs.phi_circle(X, Y, -0.5, -0.4, 0.45)
        w, ux_e, uy_e = inputs.lamb_oseen(X, Y, x0, y0, gamma, nu_t)

        def psi_lo(x, y, body=None):
            r2 = (x - x0) ** 2 + (y - y0) ** 2
            return -(gamma / (4 * math.pi)) * (np.log(r2) + exp1(r2 / (4 * nu_t)))
        P = inputs.Problem(grid=g, phi=phi, regions=[inputs.region_around(g, phi)], modes=[0],
                           omega=np.where(phi >= 0, w, 0)[1:-1, 1:-1], psi_box=inputs.box_ring(g, psi_lo(X, Y)),
                           psi_b_fn=psi_lo, psibar=np.zeros(1), gamma=None, exact=None)
        S = op.Setup(P)
        psi, pb = op.solve_unreduced(S, psibar=np.zeros(1))
        ux, uy = op.velocity(S, psi, pb)
        fl = (phi >= 0)[1:-1, 1:-1]
        errs.append(max(np.abs(ux - ux_e[1:-1, 1:-1])[fl].max(), np.abs(uy - uy_e[1:-1, 1:-1])[fl].max()))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 1.7, (errs, rates)


def test_residual_detects_perturbation():
    P = inputs.bicubic_bodies(48, seed=3, circulation=False)
    S = op.Setup(P)
    psi, pb = op.solve_unreduced(S, psibar=P.psibar)
    assert op.residual(S, psi, pb) < 1e-13
    psi2 = psi.copy()
    psi2[20, 20] += 1e-6
    assert op.residual(S, psi2, pb) > 1e-12


def test_underresolved_geometry_is_reported():
    g = inputs.square_grid(128)
    X, Y = g.nodes()
    phi = inputs.phi_star(X, Y, 0.0, 0.85, 0.5, 0.15, 5)
    geo = geom.process_geometry(g, phi, [inputs.region_around(g, phi)])
    with pytest.raises(ex.UnderResolved):
        ex.ghost_operator(geo, phi, degree=3)


def test_bad_regions_are_rejected():
    g = inputs.square_grid(64)
    X, Y = g.nodes()
    a = inputs.phi_circle(X, Y, -0.6, 0, 0.4)
    b = inputs.phi_circle(X, Y, 0.6, 0, 0.4)
    ra, rb = inputs.region_around(g, a), inputs.region_around(g, b)
    with pytest.raises(geom.GeometryError):
        geom.process_geometry(g, inputs.union(a, b), [ra])               # body b in no region
    with pytest.raises(geom.GeometryError):
        geom.process_geometry(g, a, [(ra[0] + 4, ra[1], ra[2], ra[3])])  # region cuts the body
