"""Total pressure by a Poisson problem with a Neumann wall condition (Sec. 5.4) -- oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The total pressure H = (p - p_inf) + (|u|^2 - |u_inf|^2) / 2 solves nabla^2 H = div(u x omega k)
(Eq. pressurepoisson) with the wall condition of Eq. totalpressurebc, and the solve is the IIM
Poisson solve of Sec. 4.2 with the Neumann variant of the extrapolation (Sec. 2.1).  Readings of
what the paper leaves open (each listed in the design notes):

  * Wall datum.  The Neumann extrapolation along a grid line needs the derivative of H along
    that line at the crossing, d . grad H (d the line direction pointing into the fluid), not
    only the normal part dH/dn.  On a stationary no-slip wall grad(|u|^2/2) = (grad u)^T u
    vanishes, and Eq. pressuregrad1 gives grad p = nu k x grad omega, so grad H = nu (-d_y omega,
    d_x omega): its normal part is Eq. totalpressurebc's -nu d omega / ds and its tangential
    part the nu d omega / dn of Eq. pressureflux.  On an x-line only d_y omega is needed, on a
    y-line only d_x omega: the cross-line derivative of the vorticity at the crossing.
  * That derivative uses the stencil points of the vorticity boundary condition (Sec. 5.3, as
    read in transport.vorticity_bc) on the vorticity extended at third order with omega_b:
    the values interpolated at the crossing on the next two rows (columns) combined one-sidedly
    with omega_b, both sides averaged when both are available.
  * Right-hand side.  -nabla_h^2 H = f with f = -(d_x(u_y omega) - d_y(u_x omega)) by centred
    differences of the products at fluid interior nodes; at A- nodes the third-order
    extensions (u with u_b, omega with omega_b), at and beyond the box the flow solver's box
    values (u = U_inf; omega = 0, copied from the last interior column at the right edge).
  * Surface values.  H at a control point by the quadratic through the fluid node next to the
    crossing and the next two fluid nodes on its line, evaluated at the crossing (a third-order
    extrapolation without a boundary condition, Sec. 2.1 last variant), or by the line / the
    node itself where those nodes are not fluid interior nodes.
"""
from __future__ import annotations

import numpy as np

from . import extrapolation as ex
from . import poisson as op
from . import transport as tr

PAD = tr.PAD


def pressure_rhs(T: tr.TransportSetup, omega, ux_in, uy_in, u_b, Uinf, omega_b=None):
    """f = -div(u x omega k) at fluid interior nodes (interior array, 0 in the solid) and the
    omega_b used (computed from the velocity by transport.vorticity_bc when not given)."""
    S = T.S
    h = S.h
    phi = S.prob.phi
    uxb, uyb = tr.extended_velocity(T, ux_in, uy_in, u_b, Uinf)
    if omega_b is None:
        omega_b = tr.vorticity_bc(T, uxb, uyb, u_b)
    nodes = np.zeros((S.ny + 1, S.nx + 1))
    nodes[1:-1, 1:-1] = np.where(phi[1:-1, 1:-1] >= 0, omega, 0.0)
    w3 = tr._big(S, ex.extend(nodes, phi, T.e3, omega_b), None, True)
    q = uyb * w3      # u_y omega
    r = uxb * w3      # u_x omega
    ny1, nx1 = phi.shape
    f = np.zeros((S.ny - 1, S.nx - 1))
    for j in range(1, ny1 - 1):
        for i in range(1, nx1 - 1):
            if phi[j, i] < 0:
                continue
            J, I = j + PAD, i + PAD
            dq = (q[J, I + 1] - q[J, I - 1]) / (2.0 * h)
            dr = (r[J + 1, I] - r[J - 1, I]) / (2.0 * h)
            f[j - 1, i - 1] = -(dq - dr)
    return f, omega_b


def wall_data(T: tr.TransportSetup, omega, omega_b, nu):
    """d . grad H at every control point (d along its grid line into the fluid) from
    grad H = nu (-d_y omega, d_x omega) on a stationary no-slip wall."""
    S = T.S
    h = S.h
    phi = S.prob.phi
    solid = phi < 0
    minus = S.geo["minus"]
    ny1, nx1 = solid.shape
    cps = S.geo["cp"]
    nodes = np.zeros((S.ny + 1, S.nx + 1))
    nodes[1:-1, 1:-1] = np.where(phi[1:-1, 1:-1] >= 0, omega, 0.0)
    W = tr._big(S, ex.extend(nodes, phi, T.e3, omega_b), None, True)

    def defined(i, j):
        if i <= 0 or j <= 0 or i >= nx1 - 1 or j >= ny1 - 1:
            return True
        return (not solid[j, i]) or minus[j, i]

    out = np.zeros(len(cps["t"]))
    for c in range(len(out)):
        si, sj, fi, fj, t = cps["si"][c], cps["sj"][c], cps["fi"][c], cps["fj"][c], cps["t"][c]
        di, dj = fi - si, fj - sj
        along_x = di != 0
        wb = omega_b[c]
        ests, first_order = [], None
        for s in (1, -1):
            vals, ok = [], True
            for k in (1, 2):
                pi_, pj_ = (0, k * s) if along_x else (k * s, 0)
                pts = [(si + pi_, sj + pj_), (fi + pi_, fj + pj_), (fi + di + pi_, fj + dj + pj_)]
                if not all(defined(a, b) for a, b in pts):
                    ok = False
                    break
                Wm, W0, Wp = (W[b + PAD, a + PAD] for a, b in pts)
                vals.append(W0 + (-t) * (Wp - Wm) / 2.0 + t * t * (Wp - 2.0 * W0 + Wm) / 2.0)
                if k == 1 and first_order is None:
                    first_order = s * (vals[0] - wb) / h
            if ok:
                ests.append(s * (-3.0 * wb + 4.0 * vals[0] - vals[1]) / (2.0 * h))
        d_cross = float(np.mean(ests)) if ests else (first_order if first_order is not None else 0.0)
        # x-line: d_y omega; d . grad H = di * (-nu d_y omega).  y-line: d_x omega; dj * nu d_x omega
        out[c] = -nu * di * d_cross if along_x else nu * dj * d_cross
    return out


def wall_values(S: op.Setup, field):
    """Field (interior array) extrapolated to every control point (reading above)."""
    cps = S.geo["cp"]
    solid = S.solid
    ny1, nx1 = solid.shape
    nodes = np.zeros((S.ny + 1, S.nx + 1))
    nodes[1:-1, 1:-1] = field

    def fluid_interior(i, j):
        return 1 <= i <= nx1 - 2 and 1 <= j <= ny1 - 2 and not solid[j, i]

    out = np.zeros(len(cps["t"]))
    for c in range(len(out)):
        si, sj, fi, fj, t = cps["si"][c], cps["sj"][c], cps["fi"][c], cps["fj"][c], cps["t"][c]
        di, dj = fi - si, fj - sj
        # positions along the line from the fluid node: 0 (node), 1, 2 (further into the fluid);
        # the crossing sits at -t
        pos, vals = [0.0], [nodes[fj, fi]]
        for m in (1, 2):
            a, b = fi + m * di, fj + m * dj
            if not fluid_interior(a, b):
                break
            pos.append(float(m))
            vals.append(nodes[b, a])
        w = ex.lagrange_at(pos, -t)
        out[c] = float(np.dot(w, vals))
    return out


def total_pressure(T: tr.TransportSetup, S_neumann: op.Setup, omega, ux_in, uy_in, Uinf, nu, H_box=None,
                   outer="dirichlet", tol=1e-13, u_b=None):
    """The whole Sec. 5.4 global method: right-hand side and wall data from the flow, the IIM
    solve with the Neumann wall, surface values.  Returns (H node array, H at the control points,
    f, wall data, omega_b, GMRES iterations)."""
    S = T.S
    ncp = len(S.geo["cp"]["t"])
    if u_b is None:
        u_b = (np.zeros(ncp), np.zeros(ncp))
    f, omega_b = pressure_rhs(T, omega, ux_in, uy_in, u_b, Uinf)
    data = wall_data(T, omega, omega_b, nu)
    S_neumann.psi_b = data
    ring = np.zeros(2 * (S.nx + S.ny)) if H_box is None else H_box
    H, _, it, _ = op.solve_schur(S_neumann, omega=f, ring=ring, psibar=np.zeros(S.nb), tol=tol, outer=outer)
    Hw = wall_values(S_neumann, H[1:-1, 1:-1])
    return H, Hw, f, data, omega_b, it
