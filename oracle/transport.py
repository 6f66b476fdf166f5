"""Vorticity transport on the IIM grid (Sec. 3, Sec. 5.1, 5.3, 5.5, App. B) -- oracle.

Readings of the paper used here (each listed in the design notes):
  * Advective flux (Eq. upwind): the face velocity u_{i+1/2} = (u_i + u_{i+1})/2 only selects
    the stencil; the interpolated quantity is the point flux f_j = u_j w_j (the printed product
    max(u,0) * [...] is read as the upwind indicator, since [...] already carries u).
  * Boundary faces (one side solid): when the face velocity points from the solid side into
    the fluid the downwind stencil is used instead (Sec. 3.2); at solid stencil nodes the
    vorticity extended WITH omega_b is used on the upwind side of the face and the extension
    WITHOUT a boundary condition on the downwind side (Fig. 4 caption).
  * Extensions: diffusion uses the fourth-order extension with omega_b (degree 3); advection
    the third-order ones (degree 2) with and without omega_b; velocity the third-order one with
    u_b (Sec. 3.2, 5.3).
  * Vorticity boundary condition (Sec. 5.3; its stencil figure is missing): at a control point
    on an x-line, d(u_y)/dx is the derivative at the crossing of the quadratic through the
    extended u_y at the solid node, the fluid node and the next fluid node on the line;
    d(u_x)/dy is one-sided: u_x is interpolated at the crossing's abscissa on the two rows
    j+s, j+2s by the same three-node quadratics, and combined with u_b,x at the crossing,
    (-3 u_b + 4 v1 - v2) / (2h) * s; both sides s = +1, -1 are averaged when both rows pairs
    are available (every node fluid, box or A-), one side is used when only it is; with
    neither, a first-order difference with one row, else 0.  y-lines: x and y swapped.
    Pinned by what the paper fixes, second order: exact for quadratic velocity, second-order
    convergent at every control point on the exact Lamb-Oseen field (tests).
  * Box (the Dirichlet box replaces the paper's free-space / outflow conditions): velocity
    Uinf at and beyond the box; vorticity 0 at and beyond the box except at the right
    (outflow) edge, where it is copied from the last interior column (zero gradient).
  * Low-storage RK3 of Williamson (1980): A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15).
  * Time step (App. B): dt_max from the RK3 polygon (0,0), (1.620,0), (0,0.314) in the
    (C_2D, r) plane: 1/dt_max = max(|u_x|+|u_y|)/(1.620 h) + nu/(0.314 h^2).
"""
from __future__ import annotations

import numpy as np

from . import extrapolation as ex
from . import poisson as op

RK3_A = (0.0, -5.0 / 9.0, -153.0 / 128.0)
RK3_B = (1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0)
RK3_C = (0.0, 1.0 / 3.0, 3.0 / 4.0)
STAB_C, STAB_R = 1.620, 0.314
PAD = 2   # layers beyond the box in the extended arrays


def dt_max(ux, uy, nu, h, mask=None):
    """Largest stable RK3 step on the App. B polygon edge (C_2D/1.620 + r/0.314 = 1)."""
    s = np.abs(ux) + np.abs(uy)
    if mask is not None:
        s = np.where(mask, s, 0.0)
    U = float(s.max()) if s.size else 0.0
    return 1.0 / (U / (STAB_C * h) + nu / (STAB_R * h * h))


class TransportSetup:
    """Ghost operators of the four extensions used by the transport step."""

    def __init__(self, S: op.Setup):
        self.S = S
        phi = S.prob.phi
        self.e4 = S.ghosts                                                  # degree 3 with BC
        self.e3 = ex.ghost_operator(S.geo, phi, degree=2, with_bc=True)     # degree 2 with BC
        self.e3n = ex.ghost_operator(S.geo, phi, degree=2, with_bc=False)   # degree 2, no BC


def _big(S, interior_nodes_field, box_val, right_copy):
    """(ny+1+2P) x (nx+1+2P) array: node field in the middle, box and beyond filled."""
    ny1, nx1 = interior_nodes_field.shape
    out = np.zeros((ny1 + 2 * PAD, nx1 + 2 * PAD))
    out[PAD:PAD + ny1, PAD:PAD + nx1] = interior_nodes_field
    core = out[PAD:PAD + ny1, PAD:PAD + nx1]
    if box_val is not None:
        # everything outside the interior takes box_val (velocity: Uinf)
        out[:, :] = box_val
        out[PAD + 1:PAD + ny1 - 1, PAD + 1:PAD + nx1 - 1] = interior_nodes_field[1:-1, 1:-1]
    else:
        core[0, :] = 0.0
        core[-1, :] = 0.0
        core[:, 0] = 0.0
        core[:, -1] = 0.0
        if right_copy:
            for k in range(PAD + 1):
                out[PAD + 1:PAD + ny1 - 1, PAD + nx1 - 1 + k] = interior_nodes_field[1:-1, -2]
    return out


def extended_velocity(T: TransportSetup, ux_in, uy_in, u_b, Uinf):
    """Interior-array velocity -> node arrays with E3 ghosts (with u_b) at A- and Uinf at the box."""
    S = T.S
    ny, nx = S.ny, S.nx
    out = []
    for comp, uin in enumerate((ux_in, uy_in)):
        nodes = np.zeros((ny + 1, nx + 1))
        nodes[1:-1, 1:-1] = uin
        e = ex.extend(nodes, S.prob.phi, T.e3, u_b[comp])
        out.append(_big(S, e, Uinf[comp], False))
    return out


def vorticity_bc(T: TransportSetup, uxb, uyb, u_b):
    """omega_b at every control point (Sec. 5.3) from the extended velocity (big arrays)."""
    S = T.S
    h = S.h
    cps = S.geo["cp"]
    solid = S.prob.phi < 0
    minus = S.geo["minus"]
    ny1, nx1 = solid.shape

    def defined(i, j):
        if i <= 0 or j <= 0 or i >= nx1 - 1 or j >= ny1 - 1:
            return True            # box nodes carry Uinf
        return (not solid[j, i]) or minus[j, i]

    def val(arr, i, j):
        return arr[j + PAD, i + PAD]

    wb = np.zeros(len(cps["t"]))
    for c in range(len(wb)):
        si, sj, fi, fj, t = cps["si"][c], cps["sj"][c], cps["fi"][c], cps["fj"][c], cps["t"][c]
        di, dj = fi - si, fj - sj
        along_x = di != 0
        # along-line derivative of the cross component
        A = uyb if along_x else uxb            # d(u_y)/dx on x-lines, d(u_x)/dy on y-lines
        dsgn = di if along_x else dj
        Us, Uf = val(A, si, sj), val(A, fi, fj)
        if defined(fi + di, fj + dj) and not (0 < fi + di < nx1 - 1 and 0 < fj + dj < ny1 - 1 and solid[fj + dj, fi + di]):
            Un = val(A, fi + di, fj + dj)
            d_along = dsgn / h * ((Un - Us) / 2.0 - t * (Un - 2.0 * Uf + Us))
        else:
            d_along = dsgn / h * (Uf - Us)
        # cross-line derivative of the along component, one-sided with the boundary value
        B = uxb if along_x else uyb
        ub = u_b[0][c] if along_x else u_b[1][c]
        ests = []
        first_order = None
        for s in (1, -1):
            vals = []
            ok = True
            for k in (1, 2):
                # row (x-line) or column (y-line) offset by k*s
                pi_, pj_ = (0, k * s) if along_x else (k * s, 0)
                nodes = [(si + pi_, sj + pj_), (fi + pi_, fj + pj_), (fi + di + pi_, fj + dj + pj_)]
                if not all(defined(a, b) for a, b in nodes):
                    ok = False
                    break
                Um, U0, Up = (val(B, a, b) for a, b in nodes)
                vals.append(U0 + (-t) * (Up - Um) / 2.0 + t * t * (Up - 2.0 * U0 + Um) / 2.0)
                if k == 1 and first_order is None:
                    first_order = s * (vals[0] - ub) / h
            if ok:
                ests.append(s * (-3.0 * ub + 4.0 * vals[0] - vals[1]) / (2.0 * h))
        if ests:
            d_cross = float(np.mean(ests))
        elif first_order is not None:
            d_cross = first_order
        else:
            d_cross = 0.0
        # omega = d(u_y)/dx - d(u_x)/dy
        wb[c] = (d_along - d_cross) if along_x else (d_cross - d_along)
    return wb


def _face_fluxes(T, wbig4, wbig3, wbig3n, uxb, uyb, nu, axis):
    """Face fluxes F = f + q on every face between interior-or-box nodes along `axis`.

    Returns an array Fx[j, i] = flux at face (i+1/2, j) for node indices i = 0..nx-1 (axis 0),
    or Fy[j, i] = flux at face (i, j+1/2) for j = 0..ny-1 (axis 1), in node-array indexing."""
    S = T.S
    h = S.h
    solid = S.prob.phi < 0
    ny1, nx1 = solid.shape
    if axis == 0:
        U = uxb
        nf = (ny1, nx1 - 1)
    else:
        U = uyb
        nf = (ny1 - 1, nx1)
    F = np.zeros(nf)

    def sld(i, j):
        return 0 < i < nx1 - 1 and 0 < j < ny1 - 1 and solid[j, i]

    di, dj = (1, 0) if axis == 0 else (0, 1)
    for j in range(nf[0]):
        for i in range(nf[1]):
            a = (i, j)
            b = (i + di, j + dj)
            sa, sb = sld(*a), sld(*b)
            if sa and sb:
                continue
            ua = U[a[1] + PAD, a[0] + PAD]
            ubv = U[b[1] + PAD, b[0] + PAD]
            uf = 0.5 * (ua + ubv)
            pos = uf >= 0.0
            if sa != sb:
                inflow = (sb and not pos) or (sa and pos)
                if inflow:
                    pos = not pos            # downwind stencil at inflow boundary faces
            if pos:
                nodes = [(a[0] - di, a[1] - dj), a, b]
                wts = (-1.0 / 6.0, 5.0 / 6.0, 1.0 / 3.0)
            else:
                nodes = [a, b, (b[0] + di, b[1] + dj)]
                wts = (1.0 / 3.0, 5.0 / 6.0, -1.0 / 6.0)
            # upwind side of the face: left/below when uf >= 0
            up_left = uf >= 0.0
            f = 0.0
            for (ni, nj), wgt in zip(nodes, wts):
                left_side = (ni, nj) in ((a[0] - di, a[1] - dj), a)
                if sld(ni, nj):
                    src = wbig3 if (left_side == up_left) else wbig3n
                else:
                    src = wbig3
                f += wgt * U[nj + PAD, ni + PAD] * src[nj + PAD, ni + PAD]
            q = -nu * (wbig4[b[1] + PAD, b[0] + PAD] - wbig4[a[1] + PAD, a[0] + PAD]) / h
            F[j, i] = f + q
    return F


def transport_rhs(T: TransportSetup, omega, ux_in, uy_in, u_b, Uinf, nu, omega_b=None):
    """d omega / dt (interior array, 0 in the solid) and the face fluxes (Fx, Fy) of the
    conservative scheme (Eq. 2dshuconserve) with the IIM boundary treatment (Sec. 3.2)."""
    S = T.S
    h = S.h
    phi = S.prob.phi
    uxb, uyb = extended_velocity(T, ux_in, uy_in, u_b, Uinf)
    if omega_b is None:
        omega_b = vorticity_bc(T, uxb, uyb, u_b)
    nodes = np.zeros((S.ny + 1, S.nx + 1))
    nodes[1:-1, 1:-1] = np.where(phi[1:-1, 1:-1] >= 0, omega, 0.0)
    w4 = _big(S, ex.extend(nodes, phi, T.e4, omega_b), None, True)
    w3 = _big(S, ex.extend(nodes, phi, T.e3, omega_b), None, True)
    w3n = _big(S, ex.extend(nodes, phi, T.e3n, None), None, True)
    Fx = _face_fluxes(T, w4, w3, w3n, uxb, uyb, nu, 0)
    Fy = _face_fluxes(T, w4, w3, w3n, uxb, uyb, nu, 1)
    # interior node (i, j): faces Fx[j, i-1], Fx[j, i], Fy[j-1, i], Fy[j, i]
    rhs = -((Fx[1:-1, 1:] - Fx[1:-1, :-1]) + (Fy[1:, 1:-1] - Fy[:-1, 1:-1])) / h
    rhs = np.where(phi[1:-1, 1:-1] >= 0, rhs, 0.0)
    return rhs, Fx, Fy, omega_b


def kelvin_rhs(S: op.Setup, Fx, Fy):
    """d Gamma_k / dt = -h sum_{dR_k} (f + q).n (Eq. discreteKelvinChoice), all bodies."""
    h = S.h
    out = np.zeros(S.nb)
    for k, (lx, rx, ly, ry) in enumerate(S.prob.regions):
        s = Fx[ly:ry + 1, rx].sum() - Fx[ly:ry + 1, lx - 1].sum() + Fy[ry, lx:rx + 1].sum() - Fy[ly - 1, lx:rx + 1].sum()
        out[k] = -h * s
    return out


def region_flux(S: op.Setup, Fx, Fy, region):
    """h sum_{dR} (f + q).n for any grid-aligned region (Eq. sum_dR_def)."""
    lx, rx, ly, ry = region
    return S.h * (Fx[ly:ry + 1, rx].sum() - Fx[ly:ry + 1, lx - 1].sum() + Fy[ry, lx:rx + 1].sum() - Fy[ly - 1, lx:rx + 1].sum())


def rk3_step(T: TransportSetup, omega, gamma, u_b, Uinf, nu, c_stab, dt=None, psi_b=None, psi_box=None,
             psibar=None, u_b_rate=None):
    """One low-storage RK3 step (Sec. 5.5): per stage, velocity reconstruction (Sec. 4.2) with
    Gamma_k, vorticity BC, transport RHS and Kelvin RHS, then the Williamson update of (omega,
    Gamma).  With u_b_rate (du_b/dt, same layout as u_b) the wall velocity of stage s is
    u_b + c_s dt u_b_rate at the stage time t + c_s dt (a wall driven by a law in time, as in
    the convergence study of Sec. 6.1).  Returns (omega, gamma, dt, psibar)."""
    S = T.S
    P = S.prob
    fluid = P.phi[1:-1, 1:-1] >= 0
    w = np.where(fluid, omega, 0.0).astype(np.float64)
    g = np.asarray(gamma, dtype=np.float64).copy()
    dw = np.zeros_like(w)
    dg = np.zeros_like(g)
    pb = np.zeros(S.nb) if psibar is None else np.asarray(psibar, dtype=np.float64).copy()
    saved_b = S.psi_b
    if psi_b is not None:
        S.psi_b = np.asarray(psi_b, dtype=np.float64)
    ring = P.psi_box if psi_box is None else psi_box
    try:
        for s in range(3):
            psi, pb = op.solve_unreduced(S, omega=w, ring=ring, gamma=g, psibar=pb)
            ux, uy = op.velocity(S, psi, pb)
            if s == 0 and dt is None:
                dt = c_stab * dt_max(ux, uy, nu, S.h, fluid)
            ub = u_b
            if u_b_rate is not None:
                ub = (u_b[0] + RK3_C[s] * dt * u_b_rate[0], u_b[1] + RK3_C[s] * dt * u_b_rate[1])
            rhs, Fx, Fy, _ = transport_rhs(T, w, ux, uy, ub, Uinf, nu)
            grhs = kelvin_rhs(S, Fx, Fy)
            dw = RK3_A[s] * dw + dt * rhs
            dg = RK3_A[s] * dg + dt * grhs
            w = w + RK3_B[s] * dw
            g = g + RK3_B[s] * dg
    finally:
        S.psi_b = saved_b
    return w, g, dt, pb
