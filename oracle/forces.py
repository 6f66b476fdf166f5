"""Control-volume force and moment on a stationary immersed body (App. C: Noca's momentum
formulation, Eq. Fm with the tensor gamma, and the moment formulation of Eqs. Mm1 / Mm2), for
density 1, from the velocity, vorticity and streamfunction on the grid.

Test infrastructure: imported only by the tests, the smoke check and the benchmark's CPU legs.

The control volume V is the node box [lx, rx] x [ly, ry] (global node indices) minus the body;
its outer surface S is the box's four node lines, integrated with the trapezoidal rule;
derivatives on S are centred differences (the box keeps two nodes of plain fluid from the
body and from the grid box).  With D = div T = nu lap u = nu (-d omega/dy, d omega/dx) and
T = nu (grad u + grad u^T), the surface integrands are (2D, z-components for moments)
    n.gamma = |u|^2/2 n - (n.u) u - (n.u) omega (y, -x) + (x.D) n - (n.x) D + T n,
    lambda  = |u|^2/2 (x cross n) - (x cross u)(u.n) + |x|^2/2 omega (n.u)
              + |x|^2/2 (D cross n) + x cross (T n),
with x measured from the moment centre.  The time-differentiated terms are returned as the
instantaneous integrals (the caller differentiates a time series):
    A = int_V u,  B = oint_S x cross (n cross u),  P = int_V x cross u,  Q = oint_S |x|^2/2 (n cross u),
so F = -dA/dt - dB/dt + oint n.gamma and M = -dP/dt + dQ/dt + oint lambda.
The volume integrals are rewritten with the streamfunction (u = (d psi/dy, -d psi/dx)): on a
stationary no-slip body psi is constant (psi_w) and grad psi = 0, so
    A = (oint_S psi n_y, -oint_S psi n_x),
    P = -oint_S psi (x.n) + 2 int_box psi~,
where psi~ is psi in the fluid and psi_w in the body (continuously differentiable, so the
midpoint rule over the box is second order); the body's area cancels from P.
"""
from __future__ import annotations

import numpy as np


def cv_terms(nodes_u, nodes_v, nodes_w, nodes_psi, solid, psi_wall, h, x0, y0, box, nu, xbar):
    """The nine control-volume quantities (A_x, A_y, B_x, B_y, C_x, C_y, P, Q, R) on the node box
    `box` = (lx, rx, ly, ry).  nodes_*: (ny+1, nx+1) node arrays (u, v, omega, psi); solid: node
    mask; psi_wall: psi on the body; (x0, y0): coordinates of node (0, 0); xbar: moment centre.
    C = oint n.gamma, R = oint lambda."""
    lx, rx, ly, ry = box
    X = x0 + h * np.arange(nodes_u.shape[1]) - xbar[0]
    Y = y0 + h * np.arange(nodes_u.shape[0]) - xbar[1]
    out = np.zeros(9)

    def at(i, j):
        u, v, w, p = nodes_u[j, i], nodes_v[j, i], nodes_w[j, i], nodes_psi[j, i]
        ux = (nodes_u[j, i + 1] - nodes_u[j, i - 1]) / (2 * h)
        uy = (nodes_u[j + 1, i] - nodes_u[j - 1, i]) / (2 * h)
        vx = (nodes_v[j, i + 1] - nodes_v[j, i - 1]) / (2 * h)
        vy = (nodes_v[j + 1, i] - nodes_v[j - 1, i]) / (2 * h)
        wx = (nodes_w[j, i + 1] - nodes_w[j, i - 1]) / (2 * h)
        wy = (nodes_w[j + 1, i] - nodes_w[j - 1, i]) / (2 * h)
        return u, v, w, p, ux, uy, vx, vy, wx, wy

    def integrand(i, j, n):
        x, y = X[i], Y[j]
        u, v, w, p, ux, uy, vx, vy, wx, wy = at(i, j)
        nx_, ny_ = n
        T = nu * np.array([[2 * ux, uy + vx], [uy + vx, 2 * vy]])
        D = nu * np.array([-wy, wx])
        un = nx_ * u + ny_ * v
        q = 0.5 * (u * u + v * v)
        nxu = nx_ * v - ny_ * u                      # n cross u
        Tn = T @ np.array([nx_, ny_])
        r2 = x * x + y * y
        gam = q * np.array([nx_, ny_]) - un * np.array([u, v]) - un * w * np.array([y, -x]) \
            + (x * D[0] + y * D[1]) * np.array([nx_, ny_]) - (nx_ * x + ny_ * y) * D + Tn
        lam = q * (x * ny_ - y * nx_) - (x * v - y * u) * un + 0.5 * r2 * w * un \
            + 0.5 * r2 * (D[0] * ny_ - D[1] * nx_) + (x * Tn[1] - y * Tn[0])
        return np.array([p * ny_, -p * nx_, nxu * y, -nxu * x, gam[0], gam[1],
                         -p * (x * nx_ + y * ny_), 0.5 * r2 * nxu, lam])

    # four edges, trapezoidal weights (corners at half weight on each of their two edges)
    edges = [([(i, ly) for i in range(lx, rx + 1)], (0.0, -1.0)),
             ([(i, ry) for i in range(lx, rx + 1)], (0.0, 1.0)),
             ([(lx, j) for j in range(ly, ry + 1)], (-1.0, 0.0)),
             ([(rx, j) for j in range(ly, ry + 1)], (1.0, 0.0))]
    acc = np.zeros(9)
    for pts, n in edges:
        for k, (i, j) in enumerate(pts):
            wgt = 0.5 if k in (0, len(pts) - 1) else 1.0
            acc += wgt * h * integrand(i, j, n)
    # A = (acc0, acc1); B; C; P = acc6 + 2 int_box psi~; Q; R
    out[:] = acc[[0, 1, 2, 3, 4, 5, 6, 7, 8]]
    pt = np.where(solid, psi_wall, nodes_psi)[ly:ry + 1, lx:rx + 1]
    wts = np.ones_like(pt)
    wts[0, :] *= 0.5
    wts[-1, :] *= 0.5
    wts[:, 0] *= 0.5
    wts[:, -1] *= 0.5
    out[6] += 2.0 * h * h * (wts * pt).sum()
    return out


def force_moment(terms_series, dt):
    """F = -dA/dt - dB/dt + C and M = -dP/dt + dQ/dt + R at the middle of three equally spaced
    evaluations (central difference)."""
    a, b, c = (np.asarray(t) for t in terms_series)
    d = (c - a) / (2 * dt)
    F = -d[0:2] - d[2:4] + b[4:6]
    M = -d[6] + d[7] + b[8]
    return F, M
