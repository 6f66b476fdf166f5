"""Pins of the oracle's free-space (unbounded) rectangular solve and of the free-space IIM solve
(Sec. 4.1 unbounded domains, Sec. 4.2 nabla_h^-2 with unbounded conditions, Sec. 4.3 test)."""
import math

import numpy as np
import pytest

from oracle import lgf
from oracle import poisson as op
from paper_2109_13628_gb300 import inputs


def test_lattice_green_function_closed_forms():
    """G(0,0) = 0 (gauge); -L G = delta at the origin with the lattice symmetry gives
    G(1,0) = -1/4; G(1,1) = -1/pi is the classical closed form of the potential kernel."""
    T = lgf.lgf_table(4, 4)
    assert T[0, 0] == 0.0
    assert abs(T[0, 1] + 0.25) < 1e-14 and abs(T[1, 0] + 0.25) < 1e-14
    assert abs(T[1, 1] + 1.0 / math.pi) < 1e-14
    assert abs(lgf.lgf_quad(1, 1) + 1.0 / math.pi) < 1e-13


def test_lattice_green_function_is_the_inverse_of_the_five_point_stencil():
    """-(sum of the four neighbours - 4 centre) of G is 1 at the origin and 0 elsewhere."""
    M = 40
    T = lgf.lgf_table(M + 1, M + 1)
    G = lambda m, n: T[abs(n), abs(m)]
    for m in range(0, M):
        for n in (0, 1, 3, 17, M - 1):
            L = G(m + 1, n) + G(m - 1, n) + G(m, n + 1) + G(m, n - 1) - 4.0 * G(m, n)
            assert abs(-L - (1.0 if m == n == 0 else 0.0)) < 1e-13, (m, n, L)


def test_lattice_green_function_far_field_and_composite_rule():
    """G = -(1/2 pi)(log r + euler_gamma + (3/2) log 2) + O(r^-2), and the composite rule
    equals scipy's adaptive quadrature."""
    T = lgf.lgf_table(64, 64)
    for m, n in ((16, 0), (20, 11), (33, 33), (64, 7), (50, 50)):
        r = math.hypot(m, n)
        lead = -(math.log(r) + 0.5772156649015329 + 1.5 * math.log(2.0)) / (2 * math.pi)
        assert abs(T[n, m] - lead) < 0.02 / r ** 2, (m, n, T[n, m] - lead)
    for m, n in ((0, 1), (2, 3), (7, 0), (12, 5), (24, 19)):
        assert abs(T[n, m] - lgf.lgf_quad(m, n)) < 1e-13


def test_free_space_solve_satisfies_the_five_point_equation_everywhere():
    """psi = poisson_free(f): -nabla_h^2 psi = f at every interior node, the box-adjacent ones
    included (their ring neighbours are the solution's own ring values), and outside the box
    too (f = 0 there): the convolution is evaluated at the nodes one layer out."""
    rng = np.random.default_rng(3)
    nx, ny, h = 32, 24, 0.1
    f = rng.normal(size=(ny - 1, nx - 1))
    psi = op.poisson_free(f, h)
    assert np.abs(op.neg_laplacian_5pt(psi, h) - f).max() < 1e-11 * np.abs(f).max() * max(1, 1 / h ** 2) * h * h
    # one more layer outside: the same convolution on a box grown by one node
    big = np.zeros((ny + 1, nx + 1))
    big[1:-1, 1:-1] = f
    psi_big = op.poisson_free(big, h)
    assert np.abs(psi_big[1:-1, 1:-1] - psi).max() < 1e-12 * np.abs(psi).max()
    ring_eq = op.neg_laplacian_5pt(psi_big, h)
    assert np.abs(ring_eq[[0, -1], :]).max() < 1e-10 and np.abs(ring_eq[:, [0, -1]]).max() < 1e-10


def test_free_space_lamb_oseen_velocity_second_order():
    """A Lamb-Oseen vortex in free space: velocity by centred differences of the free-space
    psi converges to the exact velocity at second order."""
    errs = []
    for n in (32, 64, 128):
        g = inputs.Grid(0.0, 1.0, 0.0, 1.0, n, n)
        X, Y = g.nodes()
        w, ux, uy = inputs.lamb_oseen(X, Y, 0.501, 0.501, 1.0, 0.0025)
        psi = op.poisson_free(w[1:-1, 1:-1], g.h)
        vx = (psi[2:, 1:-1] - psi[:-2, 1:-1]) / (2 * g.h)
        vy = -(psi[1:-1, 2:] - psi[1:-1, :-2]) / (2 * g.h)
        errs.append(max(np.abs(vx - ux[1:-1, 1:-1]).max(), np.abs(vy - uy[1:-1, 1:-1]).max()))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 1.8, (errs, rates)


def _free_two_bodies(n):
    P = inputs.lamb_oseen_two_bodies(n)
    S = op.Setup(P)
    gam = P.gamma
    psi, pb, it, rel = op.solve_schur(S, gamma=gam, outer="unbounded", tol=1e-13)
    return P, S, gam, psi, pb


def test_free_space_iim_residual_and_circulation():
    """The free-space IIM result satisfies the un-reduced equations (residual with the
    solution's own ring) and the discrete circulation constraint of each body."""
    P, S, gam, psi, pb = _free_two_bodies(64)
    assert op.residual(S, psi, pb, gamma=gam, outer="unbounded") < 1e-11
    for k, r in enumerate(P.regions):
        assert abs(op.discrete_circulation(psi, r) - gam[k]) < 1e-11


@pytest.mark.slow
def test_free_space_iim_lamb_oseen_two_bodies_second_order():
    """Sec. 4.3: a Lamb-Oseen vortex with two non-convex bodies in free space; the
    reconstructed velocity converges to the exact one at second order in the max norm."""
    c = inputs.FREE_SPACE_TWO_BODIES
    errs = []
    for n in (64, 128, 256):
        P, S, gam, psi, pb = _free_two_bodies(n)
        ux, uy = op.velocity(S, psi, pb)
        X, Y = P.grid.nodes()
        _, ex, ey = inputs.lamb_oseen(X, Y, c["x0"][0], c["x0"][1], c["gamma"], c["nu_t"])
        fl = (P.phi >= 0)[1:-1, 1:-1]
        errs.append(max(np.abs(ux - ex[1:-1, 1:-1])[fl].max(), np.abs(uy - ey[1:-1, 1:-1])[fl].max()))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 1.7, (errs, rates)


def test_ring_residual_identity():
    """The ring equations of the free-space system: zero for the free-space potential of
    interior sources, and exactly e on the ring for a field e harmonic inside the box (the box
    solve of a zero source with ring data e) -- what makes a ring error visible to the FP64
    residual."""
    rng = np.random.default_rng(1)
    nx, ny, h = 24, 16, 0.1
    psi = op.poisson_free(rng.normal(size=(ny - 1, nx - 1)), h)
    assert np.abs(op.ring_residual(psi)).max() < 1e-13 * np.abs(psi).max()
    e = rng.normal(size=2 * (nx + ny))
    H = op.ring_to_nodes(nx, ny, e)
    H[1:-1, 1:-1] = op.poisson_box(np.zeros((ny - 1, nx - 1)), h, e)
    assert np.abs(op.ring_residual(psi + H) - e).max() < 1e-12


# ----------------------------------------------------------------------------- outflow plane
def test_symmetric_solve_matches_brute_force_on_a_tiny_box():
    """poisson_free(sym=True) equals the double sum h^2 {sum_y [G(x - y) + G(x - y*)] f(y) +
    sum_j G(x - (nx, j)) plane_j} over every box node x, with G from scipy's adaptive quadrature
    (no table, no FFT)."""
    rng = np.random.default_rng(5)
    nx, ny, h = 6, 5, 0.3
    f = rng.normal(size=(ny - 1, nx - 1))
    plane = rng.normal(size=ny - 1)
    psi = op.poisson_free(f, h, sym=True, plane=plane)
    ref = np.zeros((ny + 1, nx + 1))
    for xj in range(ny + 1):
        for xi in range(nx + 1):
            acc = 0.0
            for yj in range(1, ny):
                for yi in range(1, nx):
                    acc += (lgf.lgf_quad(xi - yi, xj - yj) + lgf.lgf_quad(xi - (2 * nx - yi), xj - yj)) * f[yj - 1, yi - 1]
                acc += lgf.lgf_quad(xi - nx, xj - yj) * plane[yj - 1]
            ref[xj, xi] = h * h * acc
    assert np.abs(psi - ref).max() < 1e-12 * np.abs(ref).max()


def test_symmetric_solve_five_point_equation_and_even_plane():
    """The outflow variant: -nabla_h^2 psi = f at every interior node, and on the plane column
    (the right box edge) the five-point equation holds with the mirrored neighbour
    psi(nx + 1, j) = psi(nx - 1, j) and the plane's own source: psi is the even continuation
    there (d psi / dx = 0 on the plane).  The free-space solve without the image does not
    satisfy it."""
    rng = np.random.default_rng(7)
    nx, ny, h = 32, 24, 0.1
    f = rng.normal(size=(ny - 1, nx - 1))
    plane = rng.normal(size=ny - 1)
    for sym in (True, False):
        psi = op.poisson_free(f, h, sym=sym, plane=plane if sym else None)
        assert np.abs(op.neg_laplacian_5pt(psi, h) - f).max() < 1e-9
        eq = -(2 * psi[1:-1, nx - 1] + psi[2:, nx] + psi[:-2, nx] - 4 * psi[1:-1, nx]) / (h * h)
        if sym:
            assert np.abs(eq - plane).max() < 1e-9 * np.abs(f).max()
        else:
            assert np.abs(eq - plane).max() > 1e-3 * np.abs(f).max()


def test_symmetric_ring_residual_identity():
    """The ring equations with the symmetric kernel: zero for the outflow-variant field (its
    plane sources given), exactly e for a field e harmonic inside the box added to it; the
    free-space kernel does not give zero for the symmetric field."""
    rng = np.random.default_rng(2)
    nx, ny, h = 24, 16, 0.1
    plane = rng.normal(size=ny - 1)
    psi = op.poisson_free(rng.normal(size=(ny - 1, nx - 1)), h, sym=True, plane=plane)
    assert np.abs(op.ring_residual(psi, sym=True, plane=plane, h=h)).max() < 1e-12 * np.abs(psi).max()
    assert np.abs(op.ring_residual(psi)).max() > 1e-3 * np.abs(psi).max()
    e = rng.normal(size=2 * (nx + ny))
    H = op.ring_to_nodes(nx, ny, e)
    H[1:-1, 1:-1] = op.poisson_box(np.zeros((ny - 1, nx - 1)), h, e)
    assert np.abs(op.ring_residual(psi + H, sym=True, plane=plane, h=h) - e).max() < 1e-12


def test_symmetric_lamb_oseen_with_image_second_order():
    """A Lamb-Oseen vortex near the outflow plane x = 1 (the right edge of [0, 1]^2): the
    vorticity is the vortex plus its mirror image (even about the plane), given on the interior
    nodes and on the plane column; the outflow-variant velocity converges at second order to the
    exact velocity of the pair."""
    errs = []
    x0, y0, gam, nut = 0.8, 0.501, 1.0, 0.0025
    for n in (32, 64, 128):
        g = inputs.Grid(0.0, 1.0, 0.0, 1.0, n, n)
        X, Y = g.nodes()
        w1, ux1, uy1 = inputs.lamb_oseen(X, Y, x0, y0, gam, nut)
        w2, ux2, uy2 = inputs.lamb_oseen(X, Y, 2.0 - x0, y0, gam, nut)
        w = w1 + w2
        psi = op.poisson_free(w[1:-1, 1:-1], g.h, sym=True, plane=w[1:-1, -1])
        vx = (psi[2:, 1:-1] - psi[:-2, 1:-1]) / (2 * g.h)
        vy = -(psi[1:-1, 2:] - psi[1:-1, :-2]) / (2 * g.h)
        errs.append(max(np.abs(vx - (ux1 + ux2)[1:-1, 1:-1]).max(), np.abs(vy - (uy1 + uy2)[1:-1, 1:-1]).max()))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 1.8, (errs, rates)


def test_symmetric_iim_residual_and_circulation():
    """The IIM solve with the outflow plane (plane sources given): the result satisfies the
    un-reduced equations with the symmetric ring rows and the circulation constraint of each
    body; it is not the free-space solution."""
    P = inputs.lamb_oseen_two_bodies(64)
    S = op.Setup(P)
    plane = np.linspace(0.1, -0.2, P.grid.ny - 1)
    psi, pb, it, rel = op.solve_schur(S, gamma=P.gamma, outer="symmetric", tol=1e-13, plane=plane)
    assert op.residual(S, psi, pb, gamma=P.gamma, outer="symmetric", plane=plane) < 1e-11
    assert op.residual(S, psi, pb, gamma=P.gamma, outer="unbounded") > 1e-6
    for k, r in enumerate(P.regions):
        assert abs(op.discrete_circulation(psi, r) - P.gamma[k]) < 1e-11
