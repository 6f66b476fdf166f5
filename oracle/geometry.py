"""Geometry processing: control points (App. A), affected points (Sec. 2.2), body labels.

Reading of App. A used here (its coordinates are garbled): each control point sits on the
grid line between a solid node (phi < 0) and a fluid node (phi >= 0).  Along that line we
use the coordinate s, in units of h, measured from the fluid node towards the solid node, so
the crossing lies at t in [0, 1].  The level set restricted to the line is interpolated by a
cubic through the samples at s = -1, 0, 1, 2 (shifted to stay inside the node array at the
box edges); its root is found by Newton's method from the linear-interpolation root; if
Newton leaves [0, 1] the cubic is deflated by the Newton root and the remaining quadratic is
solved; if that also fails the linear root is kept.
"""
from __future__ import annotations

import numpy as np

X_AXIS, Y_AXIS = 0, 1


def _cubic_root(samples, s_nodes, t_lin):
    """Root in [0, 1] of the cubic interpolating samples at s_nodes (App. A)."""
    V = np.vander(np.asarray(s_nodes, dtype=np.float64), 4, increasing=True)
    a = np.linalg.solve(V, np.asarray(samples, dtype=np.float64))    # a0 + a1 s + a2 s^2 + a3 s^3

    def p(z):
        return ((a[3] * z + a[2]) * z + a[1]) * z + a[0]

    def dp(z):
        return (3.0 * a[3] * z + 2.0 * a[2]) * z + a[1]

    z = t_lin
    for _ in range(60):
        d = dp(z)
        if d == 0.0:
            break
        step = p(z) / d
        z -= step
        if abs(step) < 1e-15:
            break
    if 0.0 <= z <= 1.0:
        return z
    # deflation: p(z) = (z - z1)(b2 z^2 + b1 z + b0)
    b2 = a[3]
    b1 = a[2] + z * b2
    b0 = a[1] + z * b1
    if b2 != 0.0:
        disc = b1 * b1 - 4.0 * b2 * b0
        if disc >= 0.0:
            for r in ((-b1 + np.sqrt(disc)) / (2.0 * b2), (-b1 - np.sqrt(disc)) / (2.0 * b2)):
                if 0.0 <= r <= 1.0:
                    return float(r)
    elif b1 != 0.0:
        r = -b0 / b1
        if 0.0 <= r <= 1.0:
            return float(r)
    return t_lin


def _shifted_offsets(pos_f, step, n_line):
    """Sample offsets s = -1..2 (positions pos_f + s*step), shifted by the smallest amount
    that keeps every sample inside 0..n_line-1."""
    for k in (0, 1, -1, 2, -2):
        offs = np.arange(-1, 3) + k
        pos = pos_f + offs * step
        if pos.min() >= 0 and pos.max() <= n_line - 1:
            return offs
    raise ValueError("grid line too short for the cubic root stencil")


def control_points(grid, phi):
    """All grid-line / boundary crossings (set C, Sec. 2.2, App. A).

    Returned in canonical order: x-edges (node (i,j) to (i+1,j)) ordered by (j, i), then
    y-edges (node (i,j) to (i,j+1)) ordered by (j, i).  Fields per control point:
      axis, (i, j) of the edge's lower node, solid node (si, sj), fluid node (fi, fj),
      t = distance from the fluid node to the crossing in units of h, x, y coordinates.
    """
    ny1, nx1 = phi.shape
    solid = phi < 0
    out = {k: [] for k in ("axis", "i", "j", "si", "sj", "fi", "fj", "t", "x", "y")}
    h = grid.h
    for axis in (X_AXIS, Y_AXIS):
        di, dj = (1, 0) if axis == X_AXIS else (0, 1)
        a = solid[: ny1 - dj, : nx1 - di]
        b = solid[dj:, di:]
        js, is_ = np.nonzero(a != b)          # row-major order = ordered by (j, i)
        n_line = nx1 if axis == X_AXIS else ny1
        for j, i in zip(js.tolist(), is_.tolist()):
            if solid[j, i]:
                si, sj, fi, fj = i, j, i + di, j + dj
            else:
                si, sj, fi, fj = i + di, j + dj, i, j
            ui, uj = si - fi, sj - fj                       # unit step fluid -> solid
            pos_f = fi if axis == X_AXIS else fj
            step = ui if axis == X_AXIS else uj
            offs = _shifted_offsets(pos_f, step, n_line)
            samples = [phi[fj + o * uj, fi + o * ui] for o in offs]
            pf, ps = phi[fj, fi], phi[sj, si]
            t_lin = pf / (pf - ps)
            t = _cubic_root(samples, offs, t_lin)
            for k, v in (("axis", axis), ("i", i), ("j", j), ("si", si), ("sj", sj), ("fi", fi),
                         ("fj", fj), ("t", t), ("x", grid.x0 + h * (fi + t * ui)),
                         ("y", grid.y0 + h * (fj + t * uj))):
                out[k].append(v)
    res = {k: np.asarray(v) for k, v in out.items()}
    for k in ("axis", "i", "j", "si", "sj", "fi", "fj"):
        res[k] = res[k].astype(np.int64)
    for k in ("t", "x", "y"):
        res[k] = res[k].astype(np.float64)
    return res


def affected_points(phi):
    """Interior nodes next to a control point (set A, Sec. 2.2), split into A+ (fluid) and
    A- (solid).  Returns (mask_plus, mask_minus) as node-array booleans (box ring False)."""
    solid = phi < 0
    c = solid[1:-1, 1:-1]
    other = ((solid[1:-1, 2:] != c) | (solid[1:-1, :-2] != c)
             | (solid[2:, 1:-1] != c) | (solid[:-2, 1:-1] != c))
    plus = np.zeros_like(solid)
    minus = np.zeros_like(solid)
    plus[1:-1, 1:-1] = other & ~c
    minus[1:-1, 1:-1] = other & c
    return plus, minus


def body_of_node(regions, i, j):
    """Index of the single bounding region R_k containing node (i, j), or -1 / -2 when it is
    in none / several (Sec. 4.2: each R_k encloses one body and its affected points)."""
    hits = [k for k, (lx, rx, ly, ry) in enumerate(regions) if lx <= i <= rx and ly <= j <= ry]
    if not hits:
        return -1
    return hits[0] if len(hits) == 1 else -2


class GeometryError(ValueError):
    pass


def process_geometry(grid, phi, regions, margin_nodes=5):
    """Control points, affected points and labels; validates the bounding regions.

    Raises GeometryError when a box node is solid, when a control point comes within
    `margin_nodes` of the box (the ghost stencils would reach the box), when an affected point
    lies in no region or in several, or when a region's boundary faces are not all fluid.
    """
    solid = phi < 0
    ny1, nx1 = phi.shape
    if solid[0, :].any() or solid[-1, :].any() or solid[:, 0].any() or solid[:, -1].any():
        raise GeometryError("box nodes must be fluid")
    cps = control_points(grid, phi)
    si, sj = cps["si"], cps["sj"]
    if len(si) and (si.min() < margin_nodes or si.max() > nx1 - 1 - margin_nodes
                    or sj.min() < margin_nodes or sj.max() > ny1 - 1 - margin_nodes):
        raise GeometryError("body too close to the box")
    plus, minus = affected_points(phi)
    for (lx, rx, ly, ry) in regions:
        if lx < 2 or ly < 2 or rx > nx1 - 3 or ry > ny1 - 3 or lx > rx or ly > ry:
            raise GeometryError("region outside the interior")
        ring_in = np.zeros_like(solid)
        ring_in[ly - 1:ry + 2, lx - 1:rx + 2] = True
        ring_in[ly + 1:ry, lx + 1:rx] = False
        if (solid & ring_in).any() or ((plus | minus) & ring_in).any():
            raise GeometryError("region boundary faces must lie in non-affected fluid")
    cp_body = np.array([body_of_node(regions, a, b) for a, b in zip(si, sj)], dtype=np.int64)
    aj, ai = np.nonzero(plus | minus)
    aff_body = np.array([body_of_node(regions, a, b) for a, b in zip(ai, aj)], dtype=np.int64)
    if (cp_body < 0).any() or (aff_body < 0).any():
        raise GeometryError("affected point in no region or in several")
    return {"cp": cps, "cp_body": cp_body, "plus": plus, "minus": minus,
            "aff_i": ai.astype(np.int64), "aff_j": aj.astype(np.int64), "aff_body": aff_body,
            "aff_solid": solid[aj, ai]}
