"""Polynomial-extrapolation IIM (Sec. 2.1) and its 2D form (Sec. 2.2).

A ghost value at an outer affected point g in A- is produced, along each grid direction d
whose first node g+d is fluid, by the Lagrange polynomial through the boundary point x_alpha
(carrying the Dirichlet datum) and the fluid nodes g+2d, g+3d, ... evaluated at g; the
fluid node x_i = g+d next to the boundary is left out of the stencil (Sec. 2.1, one-sided
stencil discussion).  A direction is usable only when all its fluid nodes exist without
crossing another control point (Sec. 2.2, nonconvex fallback); the ghost is the plain mean
over usable directions (Sec. 2.2, averaging).  Degree p-1 gives an extension of order p.
The variant without a boundary condition replaces x_alpha by x_i (Sec. 2.1, last variant).
The Neumann variant (Sec. 2.1) keeps the same fluid nodes g+2d, g+3d, g+4d and replaces the
boundary value by the derivative along the line at x_alpha: the cubic p with p(m) = f(g+md),
m = 2, 3, 4, and p'(1 - t) = h * (d . grad f)(x_alpha), evaluated at g.  Its weights come from
solving that 4 x 4 system for the monomial coefficients.

Weights come from the Lagrange basis written out directly (independent of any Neville
recursion).  Positions along the line are in units of h measured from g: the boundary point
sits at 1 - t (t = distance from g+d to the crossing), the fluid nodes at 2, 3, 4, ...
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

DIRS = ((1, 0), (-1, 0), (0, 1), (0, -1))


def lagrange_at(nodes, x):
    """Values at x of the Lagrange basis polynomials of the given nodes."""
    w = []
    for m, sm in enumerate(nodes):
        v = 1.0
        for l, sl in enumerate(nodes):
            if l != m:
                v *= (x - sl) / (sm - sl)
        w.append(v)
    return np.array(w)


class UnderResolved(ValueError):
    pass


def cp_index_map(cps, shape):
    """(axis, i, j) of an edge -> control point index."""
    m = {}
    for k in range(len(cps["t"])):
        m[(int(cps["axis"][k]), int(cps["i"][k]), int(cps["j"][k]))] = k
    return m


def ghost_operator(geo, phi, degree=3, with_bc=True):
    """Ghost values at every A- node as sparse operators.

    Returns (minus_nodes, Gpsi, Gbc, n_valid):
      minus_nodes  list of (i, j) of the A- nodes (row-major order),
      Gpsi         sparse (n_minus x n_nodes) acting on the flattened node array,
      Gbc          sparse (n_minus x n_control) acting on the boundary data at control points,
      n_valid      number of usable directions per A- node.
    ghost = Gpsi @ psi_nodes.ravel() + Gbc @ data_at_control_points.
    """
    solid = phi < 0
    ny1, nx1 = phi.shape
    cps = geo["cp"]
    cmap = cp_index_map(cps, phi.shape)
    mj, mi = np.nonzero(geo["minus"])
    rows_p, cols_p, vals_p = [], [], []
    rows_b, cols_b, vals_b = [], [], []
    n_valid = np.zeros(len(mi), dtype=np.int64)
    need = degree if with_bc else degree + 1         # fluid nodes used along the line
    for r, (gi, gj) in enumerate(zip(mi.tolist(), mj.tolist())):
        entries = []
        for di, dj in DIRS:
            if solid[gj + dj, gi + di]:
                continue
            # control point on the edge between g and g+d
            axis = 0 if di != 0 else 1
            ei, ej = min(gi, gi + di), min(gj, gj + dj)
            c = cmap[(axis, ei, ej)]
            first = 2 if with_bc else 1
            ms = list(range(first, first + need))
            ok = True
            for m in ms:
                qi, qj = gi + m * di, gj + m * dj
                if not (1 <= qi <= nx1 - 2 and 1 <= qj <= ny1 - 2) or solid[qj, qi]:
                    ok = False
                    break
            if not ok:
                continue
            if with_bc:
                nodes = [1.0 - cps["t"][c]] + [float(m) for m in ms]
                w = lagrange_at(nodes, 0.0)
                entries.append((c, w[0], [(gi + m * di, gj + m * dj, w[1 + k]) for k, m in enumerate(ms)]))
            else:
                w = lagrange_at([float(m) for m in ms], 0.0)
                entries.append((None, 0.0, [(gi + m * di, gj + m * dj, w[k]) for k, m in enumerate(ms)]))
        if not entries:
            raise UnderResolved(f"A- node ({gi},{gj}) has no usable extrapolation direction")
        n_valid[r] = len(entries)
        inv = 1.0 / len(entries)
        for c, wb, plist in entries:
            if c is not None:
                rows_b.append(r)
                cols_b.append(c)
                vals_b.append(wb * inv)
            for qi, qj, wq in plist:
                rows_p.append(r)
                cols_p.append(qj * nx1 + qi)
                vals_p.append(wq * inv)
    n_minus = len(mi)
    Gpsi = sp.csr_matrix((vals_p, (rows_p, cols_p)), shape=(n_minus, ny1 * nx1))
    Gbc = sp.csr_matrix((vals_b, (rows_b, cols_b)), shape=(n_minus, len(cps["t"])))
    return list(zip(mi.tolist(), mj.tolist())), Gpsi, Gbc, n_valid


def hermite_weights(a, nodes=(2.0, 3.0, 4.0)):
    """Weights (w_d, w_2, w_3, w_4) with p(0) = w_d p'(a) + sum_m w_m p(m) for every cubic p:
    row 0 of the inverse of the system [p(m) = sum_k c_k m^k; p'(a) = sum_k k c_k a^(k-1)]."""
    M = np.zeros((4, 4))
    M[0] = [0.0, 1.0, 2.0 * a, 3.0 * a * a]
    for r, m in enumerate(nodes):
        M[1 + r] = [1.0, m, m * m, m ** 3]
    return np.linalg.inv(M)[0]


def ghost_operator_neumann(geo, phi, h):
    """Ghost values at every A- node for a Neumann wall (Sec. 2.1, Neumann variant; Sec. 2.2
    averaging), as sparse operators like ghost_operator.  The data at a control point is the
    derivative along its grid line pointing into the fluid, d . grad f at x_alpha; the cubic's
    derivative in units of h is h times it.  Usable directions: those of the degree-3 Dirichlet
    stencil (g+2d, g+3d, g+4d fluid interior nodes)."""
    solid = phi < 0
    ny1, nx1 = phi.shape
    cps = geo["cp"]
    cmap = cp_index_map(cps, phi.shape)
    mj, mi = np.nonzero(geo["minus"])
    rows_p, cols_p, vals_p = [], [], []
    rows_b, cols_b, vals_b = [], [], []
    n_valid = np.zeros(len(mi), dtype=np.int64)
    for r, (gi, gj) in enumerate(zip(mi.tolist(), mj.tolist())):
        entries = []
        for di, dj in DIRS:
            if solid[gj + dj, gi + di]:
                continue
            axis = 0 if di != 0 else 1
            c = cmap[(axis, min(gi, gi + di), min(gj, gj + dj))]
            ok = all(1 <= gi + m * di <= nx1 - 2 and 1 <= gj + m * dj <= ny1 - 2 and not solid[gj + m * dj, gi + m * di]
                     for m in (2, 3, 4))
            if not ok:
                continue
            w = hermite_weights(1.0 - cps["t"][c])
            entries.append((c, w[0] * h, [(gi + m * di, gj + m * dj, w[m - 1]) for m in (2, 3, 4)]))
        if not entries:
            raise UnderResolved(f"A- node ({gi},{gj}) has no usable extrapolation direction")
        n_valid[r] = len(entries)
        inv = 1.0 / len(entries)
        for c, wb, plist in entries:
            rows_b.append(r)
            cols_b.append(c)
            vals_b.append(wb * inv)
            for qi, qj, wq in plist:
                rows_p.append(r)
                cols_p.append(qj * nx1 + qi)
                vals_p.append(wq * inv)
    n_minus = len(mi)
    Gpsi = sp.csr_matrix((vals_p, (rows_p, cols_p)), shape=(n_minus, ny1 * nx1))
    Gbc = sp.csr_matrix((vals_b, (rows_b, cols_b)), shape=(n_minus, len(cps["t"])))
    return list(zip(mi.tolist(), mj.tolist())), Gpsi, Gbc, n_valid


def extend(field_nodes, phi, ghosts, bc_values):
    """Field with ghost values written at the A- nodes (interior solid nodes elsewhere 0)."""
    minus_nodes, Gpsi, Gbc, _ = ghosts
    out = np.where(phi >= 0, field_nodes, 0.0).astype(np.float64)
    g = Gpsi @ out.ravel()
    if bc_values is not None:
        g = g + Gbc @ bc_values
    for (i, j), v in zip(minus_nodes, g):
        out[j, i] = v
    return out
