"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and bench.py.

This module holds no arithmetic of the immersed interface method itself: it only builds
grids, level sets, right-hand sides, boundary data and bounding regions in the shapes of the
paper's flows (cylinders, nonconvex bodies, Lamb-Oseen / Gaussian vorticity).  Both the
oracle and the CUDA path consume what it returns; neither is imported here.

Conventions (used everywhere in this project):
  * a box [x0,x1]x[y0,y1] split into nx x ny cells of size h; nodes (i, j), i = 0..nx,
    j = 0..ny; unknowns live on interior nodes i = 1..nx-1, j = 1..ny-1;
  * node arrays have shape (ny+1, nx+1), interior arrays (ny-1, nx-1), x fastest;
  * level set phi < 0 is solid, phi >= 0 is fluid;
  * a bounding region R_k is the inclusive node box (lx, rx, ly, ry) (Sec. 3.1, Eq. sum_R_def).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Grid:
    x0: float
    x1: float
    y0: float
    y1: float
    nx: int
    ny: int

    @property
    def h(self) -> float:
        return (self.x1 - self.x0) / self.nx

    def nodes(self):
        """Node coordinates as (X, Y), each of shape (ny+1, nx+1)."""
        x = self.x0 + self.h * np.arange(self.nx + 1)
        y = self.y0 + self.h * np.arange(self.ny + 1)
        return np.meshgrid(x, y)

    def interior(self):
        X, Y = self.nodes()
        return X[1:-1, 1:-1], Y[1:-1, 1:-1]


def square_grid(n: int, half: float = 2.0) -> Grid:
    return Grid(-half, half, -half, half, n, n)


# ----------------------------------------------------------------------------- level sets
def phi_circle(X, Y, xc, yc, R):
    return np.hypot(X - xc, Y - yc) - R


def phi_ellipse(X, Y, xc, yc, a, b, angle):
    c, s = math.cos(angle), math.sin(angle)
    xr = c * (X - xc) + s * (Y - yc)
    yr = -s * (X - xc) + c * (Y - yc)
    return (np.sqrt((xr / a) ** 2 + (yr / b) ** 2) - 1.0) * min(a, b)


def phi_annulus(X, Y, xc, yc, r_in, r_out):
    r = np.hypot(X - xc, Y - yc)
    return np.maximum(r_in - r, r - r_out)


def phi_star(X, Y, xc, yc, r0=0.5, amp=0.15, petals=5):
    dx, dy = X - xc, Y - yc
    r = np.hypot(dx, dy)
    th = np.arctan2(dy, dx)
    return r - (r0 + amp * np.cos(petals * th))


def union(*phis):
    """Solid where any body is solid."""
    out = phis[0]
    for p in phis[1:]:
        out = np.minimum(out, p)
    return out


def region_around(grid: Grid, phi_body, margin: int = 3):
    """Inclusive node box around one body's solid nodes, grown by `margin` nodes beyond the
    affected layer (solid nodes grown by one node are the affected points)."""
    js, is_ = np.nonzero(phi_body < 0)
    lx = int(is_.min()) - 1 - margin
    rx = int(is_.max()) + 1 + margin
    ly = int(js.min()) - 1 - margin
    ry = int(js.max()) + 1 + margin
    return (lx, rx, ly, ry)


# ----------------------------------------------------------------------------- vorticity
def gaussian_vortices(X, Y, centers, strengths, sigma):
    """Sum of Gaussian (Lamb-Oseen shaped, Eq. lovorticity with sigma^2 = 2 nu t) vortices."""
    w = np.zeros_like(X)
    for (cx, cy), s in zip(centers, strengths):
        w += s / (2.0 * math.pi * sigma * sigma) * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * sigma * sigma))
    return w


def lamb_oseen(X, Y, x0, y0, gamma, nu_t):
    """Lamb-Oseen vorticity and velocity (Eqs. lovorticity, lovelocity)."""
    dx, dy = X - x0, Y - y0
    r2 = dx * dx + dy * dy
    w = gamma / (4.0 * math.pi * nu_t) * np.exp(-r2 / (4.0 * nu_t))
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(r2 > 0, gamma / (2.0 * math.pi * r2) * (1.0 - np.exp(-r2 / (4.0 * nu_t))), 0.0)
    return w, -f * dy, f * dx


def psi_lamb_oseen(X, Y, x0, y0, gamma, nu_t):
    """Lamb-Oseen streamfunction for u = (d psi/dy, -d psi/dx), additive constant dropped:
    psi = -(gamma / 4 pi) [ln r^2 + E1(r^2 / (4 nu t))] (r > 0)."""
    from scipy.special import exp1
    r2 = (X - x0) ** 2 + (Y - y0) ** 2
    return -(gamma / (4.0 * math.pi)) * (np.log(r2) + exp1(r2 / (4.0 * nu_t)))


def lamb_oseen_rate(X, Y, x0, y0, gamma, nu, t):
    """Time derivative of the Lamb-Oseen velocity (Eq. lovelocity) at time t."""
    dx, dy = X - x0, Y - y0
    r2 = dx * dx + dy * dy
    ft = -gamma * np.exp(-r2 / (4.0 * nu * t)) / (8.0 * math.pi * nu * t * t)
    return -ft * dy, ft * dx


def _rotated_cylinder_integral(kernel, t):
    from scipy import integrate
    from scipy import special as sp
    x_max = math.sqrt(40.0 / t)   # e^-40 beyond

    def f(x):
        j1, y1 = sp.j1(x), sp.y1(x)
        return kernel(x, j1, y1, sp) / (j1 * j1 + y1 * y1) * math.exp(-x * x * t)

    v, _ = integrate.quad(f, 0.0, x_max, limit=4000, epsabs=1e-13, epsrel=1e-11)
    return 2.0 / math.pi * v


def rotated_cylinder_vorticity(r, t):
    """Impulsively rotated cylinder (App. D, the real form of its vorticity integral), in the
    units r* = r/R, t* = nu t / R^2, omega* = omega / Omega:
    omega*(r, t) = (2/pi) int_0^inf (J0(xr) Y1(x) - J1(x) Y0(xr)) / (J1(x)^2 + Y1(x)^2) e^{-x^2 t} dx."""
    return _rotated_cylinder_integral(lambda x, j1, y1, sp: sp.j0(x * r) * y1 - j1 * sp.y0(x * r), t)


def rotated_cylinder_velocity(r, t):
    """u_theta / (Omega R) of the same flow (App. D, real form):
    u*(r, t) = 1/r + (2/pi) int_0^inf (J1(xr) Y1(x) - J1(x) Y1(xr)) / (J1(x)^2 + Y1(x)^2) e^{-x^2 t} / x dx."""
    return 1.0 / r + _rotated_cylinder_integral(lambda x, j1, y1, sp: (sp.j1(x * r) * y1 - j1 * sp.y1(x * r)) / x, t)


TRANSPORT_BODY = dict(xc=0.507, yc=0.531, r_a=0.201, r_b=0.054, theta_a=0.5, theta_b=2.4, u=(1.0, 2.0),
                      sigma0=0.06, x0=(0.257, 0.031), half=2.0, centre=0.5, c_stab=0.9)


def phi_notched_disk(X, Y, xc, yc, r_a, r_b, theta_a, theta_b):
    """Non-convex body of the transport study (Sec. 3.3 table; its figure is missing): the disk
    of radius r_a at (xc, yc) with two round notches of radius r_b centred on its rim at the
    angles theta_a and theta_b.  Negative inside the solid."""
    inside = np.hypot(X - xc, Y - yc) - r_a
    na = np.hypot(X - xc - r_a * math.cos(theta_a), Y - yc - r_a * math.sin(theta_a)) - r_b
    nb = np.hypot(X - xc - r_a * math.cos(theta_b), Y - yc - r_a * math.sin(theta_b)) - r_b
    return np.maximum(inside, np.maximum(-na, -nb))


def transported_gaussian(X, Y, nu, t):
    """Exact solution of d omega/dt + u.grad omega = nu lap omega for constant u: a Gaussian of
    initial width sigma0 at x0, carried with u and widened to sigma^2 = sigma0^2 + 2 nu t."""
    c = TRANSPORT_BODY
    s2 = c["sigma0"] ** 2 + 2.0 * nu * t
    dx = X - c["x0"][0] - c["u"][0] * t
    dy = Y - c["x0"][1] - c["u"][1] * t
    return c["sigma0"] ** 2 / s2 * np.exp(-(dx * dx + dy * dy) / (2.0 * s2))


def transport_body(n: int, nu: float) -> Problem:
    """Transport-only convergence workload (Sec. 3.3, adapted): the non-convex body of the
    paper's table in a box [-1.5, 2.5]^2 (n x n cells) crossed by a Gaussian vortex blob carried
    by the constant velocity u = (1, 2) (the paper's periodic cosine field is replaced by a
    localised exact solution because the box here is not periodic; the blob stays > 10 widths
    from the box for the integration times used)."""
    c = TRANSPORT_BODY
    g = Grid(c["centre"] - c["half"], c["centre"] + c["half"], c["centre"] - c["half"], c["centre"] + c["half"], n, n)
    X, Y = g.nodes()
    phi = phi_notched_disk(X, Y, c["xc"], c["yc"], c["r_a"], c["r_b"], c["theta_a"], c["theta_b"])
    w = transported_gaussian(X, Y, nu, 0.0)
    return Problem(grid=g, phi=phi, regions=[region_around(g, phi)], modes=[1], omega=_mask_interior(g, phi, w),
                   psi_box=np.zeros(4 * n), psi_b_fn=lambda x, y, body: np.zeros_like(x), psibar=np.zeros(1),
                   gamma=np.zeros(1), exact=None, name=f"transport_body_{n}")


# Sec. 4.3 (free-space velocity reconstruction): vortex and notched bodies of the paper's table;
# the printed centres put the two bodies 0.014 apart with interlocking bounding boxes (no
# rectangle R_k encloses one body without the other), so the bodies are moved apart here, with
# their shapes, sizes and notches kept.
FREE_SPACE_TWO_BODIES = dict(x0=(0.501, 0.501), gamma=1.0, nu_t=0.0025,
                             bodies=[dict(xc=0.26, yc=0.72, r_a=0.167, r_b=0.057, theta_a=0.5, theta_b=1.8),
                                     dict(xc=0.68, yc=0.34, r_a=0.157, r_b=0.057, theta_a=3.7, theta_b=2.0)])


def lamb_oseen_two_bodies(n: int) -> Problem:
    """Free-space reconstruction workload (Sec. 4.3, adapted as above): unit box, n x n cells,
    a Lamb-Oseen vortex (Eq. lovorticity) and two notched disks in circulation mode; the body
    data psi_b is the Lamb-Oseen streamfunction at the crossings (the velocity it implies is
    the exact u_b); Gamma_k = h^2 sum over the nodes of R_k of the original (unmasked)
    Lamb-Oseen vorticity, as in the paper (the vortex's circulation inside each body included).
    The box ring is not data in free space (psi_box zeros)."""
    c = FREE_SPACE_TWO_BODIES
    g = Grid(0.0, 1.0, 0.0, 1.0, n, n)
    X, Y = g.nodes()
    bodies = [phi_notched_disk(X, Y, b["xc"], b["yc"], b["r_a"], b["r_b"], b["theta_a"], b["theta_b"])
              for b in c["bodies"]]
    phi = union(*bodies)
    w, _, _ = lamb_oseen(X, Y, c["x0"][0], c["x0"][1], c["gamma"], c["nu_t"])

    def psi_b(x, y, body=None):
        return psi_lamb_oseen(x, y, c["x0"][0], c["x0"][1], c["gamma"], c["nu_t"])
    regions = [region_around(g, b) for b in bodies]
    gam = np.array([g.h * g.h * w[ly:ry + 1, lx:rx + 1].sum() for (lx, rx, ly, ry) in regions])
    return Problem(grid=g, phi=phi, regions=regions, modes=[1, 1], omega=_mask_interior(g, phi, w),
                   psi_box=np.zeros(4 * n), psi_b_fn=psi_b, psibar=np.zeros(2), gamma=gam, exact=None,
                   name=f"lamb_oseen_two_bodies_{n}")


ROTATED_CYLINDER = dict(R=0.5, omega=1.0, re=50.0, xc=0.013, yc=0.007, half=2.0, c_stab=0.5)


def rotated_cylinder(n: int) -> Problem:
    """Impulsively rotated cylinder (Sec. 6.2): box [-2,2]^2 with n x n cells, cylinder R = 0.5
    (centre slightly off the grid's symmetry lines), fluid at rest at t = 0, Re = R^2 Omega / nu
    = 50; the body is in circulation mode with zero psi_b and zero initial circulation.  The box
    is Dirichlet with psi = 0: the fluid's total circulation is zero at every t, so the flow at
    the box is exponentially small while the vorticity stays within a few sqrt(nu t) of the wall."""
    c = ROTATED_CYLINDER
    g = square_grid(n, c["half"])
    X, Y = g.nodes()
    phi = phi_circle(X, Y, c["xc"], c["yc"], c["R"])
    return Problem(grid=g, phi=phi, regions=[region_around(g, phi)], modes=[1], omega=np.zeros((n - 1, n - 1)),
                   psi_box=np.zeros(4 * n), psi_b_fn=lambda x, y, body: np.zeros_like(x), psibar=np.zeros(1),
                   gamma=np.zeros(1), exact=None, name=f"rotated_cylinder_{n}")


# ----------------------------------------------------------------------------- manufactured
def psi_c1(X, Y):
    """Streamfunction of the single-cylinder manufactured case: sin(pi x/2) sin(pi y/2) + 0.1 log r."""
    with np.errstate(divide="ignore"):
        return np.sin(np.pi * X / 2) * np.sin(np.pi * Y / 2) + 0.1 * np.log(np.hypot(X, Y))


def omega_c1(X, Y):
    """-Laplacian of psi_c1 (log r is harmonic away from the origin)."""
    return (np.pi ** 2 / 2) * np.sin(np.pi * X / 2) * np.sin(np.pi * Y / 2)


def bicubic_coeffs(seed: int):
    """Random coefficients c[a, b] of a polynomial sum c_ab x^a y^b with a, b <= 3."""
    rng = np.random.default_rng(seed)
    return rng.normal(size=(4, 4))


def bicubic(X, Y, c):
    out = np.zeros_like(X)
    for a in range(4):
        for b in range(4):
            out = out + c[a, b] * X ** a * Y ** b
    return out


def bicubic_neg_laplacian(X, Y, c):
    out = np.zeros_like(X)
    for a in range(4):
        for b in range(4):
            if a >= 2:
                out = out - c[a, b] * a * (a - 1) * X ** (a - 2) * Y ** b
            if b >= 2:
                out = out - c[a, b] * b * (b - 1) * X ** a * Y ** (b - 2)
    return out


def box_ring(grid: Grid, node_values):
    """Pack box-node data in the order used by the solver: bottom row j=0 (i=0..nx), top row
    j=ny (i=0..nx), left column i=0 (j=1..ny-1), right column i=nx (j=1..ny-1)."""
    v = np.asarray(node_values)
    return np.concatenate([v[0, :], v[-1, :], v[1:-1, 0], v[1:-1, -1]]).astype(np.float64)


# ----------------------------------------------------------------------------- workloads
@dataclasses.dataclass
class Problem:
    grid: Grid
    phi: np.ndarray               # (ny+1, nx+1)
    regions: list                 # [(lx, rx, ly, ry)] per body
    modes: list                   # 0 fixed psibar, 1 circulation given
    omega: np.ndarray             # (ny-1, nx-1) interior, zero in the solid
    psi_box: np.ndarray           # 2 (nx + ny) box ring
    psi_b_fn: object              # callable (x, y, body) -> psi_b at control points
    psibar: np.ndarray            # per body: given value (fixed) / expected value (circulation)
    gamma: np.ndarray | None      # per body circulation (circulation mode) or None
    exact: np.ndarray | None      # exact node-array streamfunction where known
    name: str = ""


def _mask_interior(grid, phi, field_nodes):
    w = np.where(phi >= 0, field_nodes, 0.0)
    return np.ascontiguousarray(w[1:-1, 1:-1])


def c1_cylinder(n: int = 128) -> Problem:
    """Manufactured single-cylinder problem on [-2,2]^2 with n x n cells, circle R=0.5."""
    g = square_grid(n)
    X, Y = g.nodes()
    phi = phi_circle(X, Y, 0.0, 0.0, 0.5)
    psi = psi_c1(X, Y)
    return Problem(
        grid=g, phi=phi, regions=[region_around(g, phi)], modes=[0],
        omega=_mask_interior(g, phi, omega_c1(X, Y)),
        psi_box=box_ring(g, psi),
        psi_b_fn=lambda x, y, body: psi_c1(x, y),
        psibar=np.zeros(1), gamma=None, exact=psi, name=f"c1_cylinder_{n}")


def bicubic_bodies(n: int, seed: int = 0, circulation: bool = True, offsets=(0.3, -0.7, 0.15)) -> Problem:
    """Polynomial-exactness workload: a bicubic streamfunction psi* around a cylinder, an ellipse
    and a nonconvex star.  The discrete IIM solution equals psi* at every fluid node (to
    rounding), for any n.  psi_b = psi* - offset_k so the expected body constants are offset_k."""
    g = square_grid(n)
    X, Y = g.nodes()
    bodies = [phi_circle(X, Y, -0.9, -0.8, 0.45),
              phi_ellipse(X, Y, 0.9, -0.7, 0.5, 0.3, 0.6),
              phi_star(X, Y, 0.0, 0.85, 0.55, 0.1, 4)]
    phi = union(*bodies)
    c = bicubic_coeffs(seed)
    psi = bicubic(X, Y, c)
    regions = [region_around(g, b) for b in bodies]
    offs = np.array(offsets[: len(bodies)], dtype=np.float64)
    mode = 1 if circulation else 0
    return Problem(
        grid=g, phi=phi, regions=regions, modes=[mode] * len(bodies),
        omega=_mask_interior(g, phi, bicubic_neg_laplacian(X, Y, c)),
        psi_box=box_ring(g, psi),
        psi_b_fn=lambda x, y, body: bicubic(x, y, c) - offs[body],
        psibar=offs.copy(), gamma=None, exact=psi, name=f"bicubic_{n}_s{seed}")


def separated_centers(rng, n_bodies, lo, hi, radii, gap):
    """Rejection-sample centers in [lo,hi]^2 keeping circles of the given radii `gap` apart."""
    centers = []
    for r in radii:
        for _ in range(10000):
            c = rng.uniform(lo, hi, size=2)
            if all(np.hypot(*(c - c2)) >= r + r2 + gap for c2, r2 in zip(centers, radii)):
                centers.append(c)
                break
        else:
            raise RuntimeError("could not place bodies")
    return centers


def vortex_field(g: Grid, seed: int, count: int = 50, sigma: float = 0.1, lo=None, hi=None):
    rng = np.random.default_rng(seed)
    lo = g.x0 if lo is None else lo
    hi = g.x1 if hi is None else hi
    centers = rng.uniform(lo, hi, size=(count, 2))
    strengths = rng.normal(size=count)
    X, Y = g.nodes()
    return gaussian_vortices(X, Y, centers, strengths, sigma)


def multibody(n: int = 2048, half: float = 4.0, seed: int = 0) -> Problem:
    """Multiply connected, nonconvex geometry: three circles (R in [0.3, 0.6]), an annulus
    (0.4 / 0.8) and a five-petal star, centers seeded in [-3,3]^2; 50 Gaussian vortices
    (sigma = 0.1, strengths N(0,1), seed 1).  Bodies in circulation mode with Gamma_k equal
    to the vorticity summed over R_k (zero circulation on the body itself)."""
    g = square_grid(n, half)
    X, Y = g.nodes()
    rng = np.random.default_rng(seed)
    radii_c = rng.uniform(0.3, 0.6, size=3)
    extent = list(radii_c) + [0.8, 0.65]
    centers = separated_centers(rng, 5, -3.0, 3.0, extent, 0.25)
    bodies = [phi_circle(X, Y, centers[k][0], centers[k][1], radii_c[k]) for k in range(3)]
    bodies.append(phi_annulus(X, Y, centers[3][0], centers[3][1], 0.4, 0.8))
    bodies.append(phi_star(X, Y, centers[4][0], centers[4][1], 0.5, 0.15, 5))
    phi = union(*bodies)
    w_nodes = vortex_field(g, seed + 1, 50, 0.1, -half, half)
    omega = _mask_interior(g, phi, w_nodes)
    regions = [region_around(g, b) for b in bodies]
    return Problem(grid=g, phi=phi, regions=regions, modes=[1] * 5, omega=omega,
                   psi_box=np.zeros(2 * (g.nx + g.ny)), psi_b_fn=lambda x, y, body: np.zeros_like(x),
                   psibar=np.zeros(5), gamma=None, exact=None, name=f"multibody_{n}")


def ellipses_problem(n: int, seed: int) -> Problem:
    """One batched-workload problem: [-2,2]^2, 1-4 ellipses (semi-axes in [0.2,0.6], random
    orientation), Gaussian-vortex right-hand side, circulation mode."""
    g = square_grid(n)
    X, Y = g.nodes()
    rng = np.random.default_rng(seed)
    nb = int(rng.integers(1, 5))
    axes = rng.uniform(0.2, 0.6, size=(nb, 2))
    angles = rng.uniform(0.0, math.pi, size=nb)
    gap = max(0.25, 8.0 * g.h)
    centers = separated_centers(rng, nb, -1.2, 1.2, list(axes.max(axis=1)), gap)
    bodies = [phi_ellipse(X, Y, centers[k][0], centers[k][1], axes[k, 0], axes[k, 1], angles[k]) for k in range(nb)]
    phi = union(*bodies)
    w_nodes = vortex_field(g, seed + 7, 50, 0.1)
    regions = [region_around(g, b) for b in bodies]
    return Problem(grid=g, phi=phi, regions=regions, modes=[1] * nb,
                   omega=_mask_interior(g, phi, w_nodes), psi_box=np.zeros(2 * (g.nx + g.ny)),
                   psi_b_fn=lambda x, y, body: np.zeros_like(x), psibar=np.zeros(nb), gamma=None,
                   exact=None, name=f"ellipses_{n}_s{seed}")


def c2_cylinder_flow(nx: int = 1024, ny: int = 512, seed: int = 0) -> Problem:
    """Flow past one cylinder (R = 0.5 at (-1, 0)) on [-2,6]x[-2,2], uniform inflow U = 1,
    Re = U D / nu = 200 (nu = 0.005): initial vorticity of the potential flow (zero) plus
    seeded Gaussian noise of amplitude 1e-3 at every fluid node; box streamfunction U y."""
    h = 8.0 / nx
    g = Grid(-2.0, 6.0, -2.0, -2.0 + h * ny, nx, ny)
    X, Y = g.nodes()
    phi = phi_circle(X, Y, -1.0, 0.0, 0.5)
    rng = np.random.default_rng(seed)
    noise = 1e-3 * rng.normal(size=(ny + 1, nx + 1))
    omega = _mask_interior(g, phi, noise)
    return Problem(grid=g, phi=phi, regions=[region_around(g, phi)], modes=[1], omega=omega,
                   psi_box=box_ring(g, 1.0 * Y), psi_b_fn=lambda x, y, body: np.zeros_like(x),
                   psibar=np.zeros(1), gamma=None, exact=None, name=f"c2_cylinder_flow_{nx}x{ny}")


LAMB_OSEEN_CYLINDER = dict(gamma=math.pi, nu=1e-3, xc=0.507, yc=0.507, R=0.15, t0=1.0, c_stab=0.7)


def lamb_oseen_cylinder(n: int, t: float | None = None) -> Problem:
    """Navier-Stokes convergence workload (Sec. 6.1 and its parameter table): unit box with
    n x n cells, cylinder R = 0.15 at (0.507, 0.507) whose wall moves with the velocity of a
    Lamb-Oseen vortex (Gamma = pi, nu = 1e-3) centred on it, the vortex's vorticity at time t
    (default t0 = 1) outside the cylinder.  The box is Dirichlet with the vortex streamfunction
    (at the box the vortex is potential to e^-30, so this data does not change in time); the
    body is in circulation mode with zero psi_b (the wall is a streamline)."""
    c = LAMB_OSEEN_CYLINDER
    t = c["t0"] if t is None else t
    g = Grid(0.0, 1.0, 0.0, 1.0, n, n)
    X, Y = g.nodes()
    phi = phi_circle(X, Y, c["xc"], c["yc"], c["R"])
    w, _, _ = lamb_oseen(X, Y, c["xc"], c["yc"], c["gamma"], c["nu"] * t)
    psi = psi_lamb_oseen(X, Y, c["xc"], c["yc"], c["gamma"], c["nu"] * t)
    return Problem(grid=g, phi=phi, regions=[region_around(g, phi)], modes=[1], omega=_mask_interior(g, phi, w),
                   psi_box=box_ring(g, psi), psi_b_fn=lambda x, y, body: np.zeros_like(x), psibar=np.zeros(1),
                   gamma=None, exact=psi, name=f"lamb_oseen_cylinder_{n}")


def batched_c4(count: int = 96, seed: int = 2, sizes=(128, 256, 512, 1024)):
    """Batched workload: `count` problems, grid sizes drawn uniformly from `sizes`, each with
    1-4 seeded ellipses and a Gaussian-vortex right-hand side (ellipses_problem)."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    return [ellipses_problem(int(n), seed * 1000 + k) for k, n in enumerate(ns)]
