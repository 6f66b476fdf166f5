"""IIM Poisson solve (Sec. 4.2): the discrete result, written two ways.

* ``solve_unreduced`` is the definition of the discrete result: the five-point Laplacian
  (Sec. 4.2) applied to the extended field psi_ext (fluid values, box data, and ghost values
  at A- from Sec. 2.1/2.2 with the Dirichlet data psi_b + psibar_k, Eq. psibc) must equal
  omega at every fluid interior node, and every circulation-mode body adds the discrete
  circulation constraint -h sum_{dR_k} (grad_h psi).n = Gamma_k (Eq. discretecircconstraint).
  Assembled as a sparse matrix and solved directly.
* ``solve_schur`` is the paper's algorithm: corrections gamma on the affected points
  (Eq. discretepoisson, poissoncorrections), the Schur complement in gamma plus the
  circulation rows (the augmented system at the end of Sec. 4.2), GMRES, and recovery of psi
  (Eq. psirecovery).  The rectangular solve uses a DST-I (the Dirichlet box).

Sign reading: substituting Eq. poissoncorrections and Eq. psirecovery into Eq. discretepoisson
with nabla_h^-2 the inverse of the five-point Laplacian gives (I - A nabla^-2 E_a) gamma =
-A nabla^-2 omega + B psi_b; with P = -nabla^-2 (the positive solver used here) that is
(I + A P E_a) gamma = A P omega + B psi_b.  The printed Eq. schur has the opposite sign on
the left; the two forms agree only with the sign derived here (pinned by a test against the
un-reduced solve).  Circulation rows: sum_{B_k} gamma = sum_{R_k} omega - Gamma_k / h^2 (the
h^2 of the constraint kept).

Layouts: node arrays (ny+1, nx+1); interior arrays (ny-1, nx-1); box ring as in
paper_2109_13628_gb300.inputs.box_ring.
"""
from __future__ import annotations

import numpy as np
import scipy.fft
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import extrapolation as ex
from . import geometry as geom


# ----------------------------------------------------------------------------- box data
def ring_to_nodes(nx, ny, ring):
    """Node array holding the box ring values (interior zero)."""
    out = np.zeros((ny + 1, nx + 1))
    o = 0
    out[0, :] = ring[o:o + nx + 1]; o += nx + 1
    out[-1, :] = ring[o:o + nx + 1]; o += nx + 1
    out[1:-1, 0] = ring[o:o + ny - 1]; o += ny - 1
    out[1:-1, -1] = ring[o:o + ny - 1]
    return out


# ----------------------------------------------------------------------------- Laplacian
def neg_laplacian_5pt(nodes, h):
    """-nabla_h^2 at interior nodes of a node array (Sec. 4.2, five-point stencil)."""
    c = nodes[1:-1, 1:-1]
    return (4.0 * c - nodes[1:-1, 2:] - nodes[1:-1, :-2] - nodes[2:, 1:-1] - nodes[:-2, 1:-1]) / (h * h)


# ----------------------------------------------------------------------------- DST-I
def dst1_matrix(x):
    """S(x)_k = sum_{j=1}^{N} x_j sin(pi j k / (N+1)), the sine-matrix definition (small N)."""
    N = x.shape[-1]
    j = np.arange(1, N + 1)
    M = np.sin(np.pi * np.outer(j, j) / (N + 1))
    return x @ M


def dst1(x, axis=-1):
    """Same transform via scipy's DST-I (which carries an extra factor 2)."""
    return 0.5 * scipy.fft.dst(x, type=1, axis=axis)


def eigenvalues(n, h):
    """Eigenvalues of -d^2/dx^2 (three-point, Dirichlet) for modes k = 1..n-1."""
    k = np.arange(1, n)
    return (2.0 - 2.0 * np.cos(np.pi * k / n)) / (h * h)


def poisson_box(f, h, ring=None):
    """u = P f: the solution of -nabla_h^2 u = f on the interior nodes with Dirichlet box
    data `ring` (zero when None) -- the rectangular solver written nabla_h^-2 in Sec. 4.2."""
    ny1, nx1 = f.shape
    nx, ny = nx1 + 1, ny1 + 1
    g = np.array(f, dtype=np.float64, copy=True)
    if ring is not None:
        b = ring_to_nodes(nx, ny, ring)
        g[:, 0] += b[1:-1, 0] / (h * h)
        g[:, -1] += b[1:-1, -1] / (h * h)
        g[0, :] += b[0, 1:-1] / (h * h)
        g[-1, :] += b[-1, 1:-1] / (h * h)
    F = dst1(dst1(g, axis=1), axis=0)
    lam = eigenvalues(nx, h)[None, :] + eigenvalues(ny, h)[:, None]
    U = F / lam
    return dst1(dst1(U, axis=1), axis=0) * (2.0 / nx) * (2.0 / ny)


def poisson_free(f, h, sym=False, plane=None):
    """Free-space solve (Sec. 4.1, unbounded domain; Sec. 4.2, nabla_h^-2 with unbounded
    boundary conditions): psi = h^2 sum_y G(x - y) f(y) with the lattice Green's function G of
    the five-point Laplacian (oracle/lgf.py, gauge G(0, 0) = 0), for f on the interior nodes.
    Returns psi at every node of the box, interior and ring: a node array (ny+1, nx+1).  The
    convolution is a plain zero-padded linear convolution (scipy's FFT convolution).

    sym: the outflow variant of Sec. 5.2 -- the vorticity mirrored evenly across the vertical
    plane through the right box edge (node column nx): the sources are f on the interior nodes,
    their images at y* = (2 nx - i, j), and `plane` (ny - 1 values, rows 1..ny-1; zero if None)
    on the plane column itself, which is its own image:
        psi(x) = h^2 { sum_y [G(x - y) + G(x - y*)] f(y) + sum_j G(x - (nx, j)) plane_j }.
    psi is then even about the plane (d psi / dx = 0 there, so u_y = 0 and d u_x / dx = 0)."""
    from scipy.signal import fftconvolve

    from . import lgf
    ny1, nx1 = f.shape
    nx, ny = nx1 + 1, ny1 + 1
    if not sym:
        src = np.zeros((ny + 1, nx + 1))
        src[1:-1, 1:-1] = f
        full = fftconvolve(src, lgf.lgf_full(nx, ny), mode="full")
        return h * h * full[ny:2 * ny + 1, nx:2 * nx + 1]
    W = 2 * nx                      # source columns 0..2nx: the box, the plane and the image
    src = np.zeros((ny + 1, W + 1))
    src[1:-1, 1:nx] = f
    src[1:-1, W - nx + 1:W] = f[:, ::-1]    # column 2nx - i holds f(i)
    if plane is not None:
        src[1:-1, nx] = plane
    full = fftconvolve(src, lgf.lgf_full(W, ny), mode="full")
    return h * h * full[ny:2 * ny + 1, W:W + nx + 1]


def plane_potential(nx, ny, h, plane):
    """h^2 sum_j G(x - (nx, j)) plane_j on the box ring (ring layout): the field of the sources
    on the outflow plane, harmonic inside the box."""
    from . import lgf
    G = lgf.lgf_table(nx + 1, ny + 1)
    ring = [(i, 0) for i in range(nx + 1)] + [(i, ny) for i in range(nx + 1)] + \
           [(0, j) for j in range(1, ny)] + [(nx, j) for j in range(1, ny)]
    js = np.arange(1, ny)
    return np.array([h * h * (G[np.abs(xj - js), abs(xi - nx)] * plane).sum() for xi, xj in ring])


def ring_of(nodes):
    """The box ring (layout of ring_to_nodes) of a node array."""
    return np.concatenate([nodes[0, :], nodes[-1, :], nodes[1:-1, 0], nodes[1:-1, -1]])


def ring_residual(nodes, sym=False, plane=None, h=None):
    """Free-space consistency of the box ring: for a field that is the free-space potential of
    sources inside the box, the discrete Green's second identity on the interior nodes (the
    five-point stencil summed by parts against G(x - .), which is harmonic there for x on the
    ring) gives psi(x) = sum over the non-corner ring nodes z of G(x - z) psi(n(z)) -
    G(x - n(z)) psi(z), n(z) the interior neighbour of z.  Returns psi(x) minus that sum on the
    ring (ring layout): zero for free-space fields, exactly e(x) for a field e harmonic inside
    the box.

    sym (the outflow variant, see poisson_free): the kernel is K(x, y) = G(x - y) + G(x* - y),
    x* = (2 nx - i, j) the image of the ring node x across the right box edge.  The mirrored
    part of the field is harmonic inside the box and G(x* - .) is harmonic there too, so the
    same identity holds with K: psi(x) = psi_f(x) + psi_f(x*) = sum K(x, z) psi(n(z)) -
    K(x, n(z)) psi(z).  Sources on the plane column (`plane`, with the grid spacing h) make a
    field harmonic inside the box, which the identity leaves on the ring: it is subtracted
    (plane_potential)."""
    from . import lgf
    ny, nx = nodes.shape[0] - 1, nodes.shape[1] - 1
    G = lgf.lgf_table(2 * nx + 1 if sym else nx + 1, ny + 1)
    ring = [(i, 0) for i in range(nx + 1)] + [(i, ny) for i in range(nx + 1)] + \
           [(0, j) for j in range(1, ny)] + [(nx, j) for j in range(1, ny)]
    src = [((i, 0), (i, 1)) for i in range(1, nx)] + [((i, ny), (i, ny - 1)) for i in range(1, nx)] + \
          [((0, j), (1, j)) for j in range(1, ny)] + [((nx, j), (nx - 1, j)) for j in range(1, ny)]
    zi = np.array([z[0] for z, _ in src]); zj = np.array([z[1] for z, _ in src])
    ai = np.array([a[0] for _, a in src]); aj = np.array([a[1] for _, a in src])

    def K(xi, xj, yi, yj):
        k = G[np.abs(xj - yj), np.abs(xi - yi)]
        if sym:
            k = k + G[np.abs(xj - yj), np.abs(2 * nx - xi - yi)]
        return k

    out = np.empty(len(ring))
    for t, (xi, xj) in enumerate(ring):
        s = (K(xi, xj, zi, zj) * nodes[aj, ai]).sum() - (K(xi, xj, ai, aj) * nodes[zj, zi]).sum()
        out[t] = nodes[xj, xi] - s
    if sym and plane is not None:
        out = out - plane_potential(nx, ny, h, plane)
    return out


# ----------------------------------------------------------------------------- setup
class Setup:
    """Geometry, ghost operators and index maps of one problem (Sec. 2.2, App. A)."""

    def __init__(self, prob, degree=3, wall="dirichlet", wall_data=None):
        """wall = "dirichlet": psi = psi_b + psibar_k on the bodies (Sec. 4.2).  wall = "neumann":
        the Neumann variant of the extrapolation (Sec. 2.1, used by the total-pressure problem of
        Sec. 5.4); the data at each control point is the derivative along its grid line into the
        fluid (wall_data, else prob.psi_b_fn), every body has fixed mode and psibar = 0."""
        self.prob = prob
        g = prob.grid
        self.nx, self.ny, self.h = g.nx, g.ny, g.h
        self.wall = wall
        self.geo = geom.process_geometry(g, prob.phi, prob.regions)
        if wall == "dirichlet":
            self.ghosts = ex.ghost_operator(self.geo, prob.phi, degree=degree, with_bc=True)
        elif wall == "neumann":
            if any(m != 0 for m in prob.modes):
                raise ValueError("a Neumann wall has no circulation unknowns: every body must be fixed")
            self.ghosts = ex.ghost_operator_neumann(self.geo, prob.phi, g.h)
        else:
            raise ValueError(wall)
        self.solid = prob.phi < 0
        cps = self.geo["cp"]
        self.cp_body = self.geo["cp_body"]
        if wall_data is not None:
            self.psi_b = np.asarray(wall_data, dtype=np.float64)
        else:
            self.psi_b = np.asarray(prob.psi_b_fn(cps["x"], cps["y"], self.cp_body), dtype=np.float64)
        self.modes = list(prob.modes)
        self.nb = len(prob.regions)
        self.circ = [k for k in range(self.nb) if self.modes[k] == 1]

    def bc_values(self, psibar):
        return self.psi_b + np.asarray(psibar)[self.cp_body]


def discrete_circulation(nodes, region):
    """-h sum_{dR}(grad_h psi).n (Eq. sum_dR_def applied to the flux (psi_{i+1}-psi_i)/h)."""
    lx, rx, ly, ry = region
    s = (nodes[ly:ry + 1, rx + 1] - nodes[ly:ry + 1, rx]).sum()
    s += (nodes[ry + 1, lx:rx + 1] - nodes[ry, lx:rx + 1]).sum()
    s -= (nodes[ly:ry + 1, lx] - nodes[ly:ry + 1, lx - 1]).sum()
    s -= (nodes[ly, lx:rx + 1] - nodes[ly - 1, lx:rx + 1]).sum()
    return -s


def region_sum(interior, region):
    """sum_R over interior-array values (Eq. sum_R_def without the h^2)."""
    lx, rx, ly, ry = region
    return interior[ly - 1:ry, lx - 1:rx].sum()


def gamma_from_regions(prob):
    """Gamma_k = h^2 sum_{R_k} omega: zero circulation on each body itself (Eq. circregion)."""
    h = prob.grid.h
    return np.array([h * h * region_sum(prob.omega, r) for r in prob.regions])


# ----------------------------------------------------------------------------- un-reduced system
def assemble_unreduced(S: Setup, omega, ring, gamma, psibar_fixed):
    """Sparse un-reduced system L u = f.  Unknowns: psi at fluid interior nodes (row-major),
    then psibar_k of each circulation-mode body.  Circulation rows are divided by h^2 so
    that every row is in the units of omega."""
    nx, ny, h = S.nx, S.ny, S.h
    nx1 = nx + 1
    solid = S.solid
    inner = np.zeros_like(solid)
    inner[1:-1, 1:-1] = True
    fluid_in = inner & ~solid
    idx = -np.ones(solid.shape, dtype=np.int64)
    nf = int(fluid_in.sum())
    idx[fluid_in] = np.arange(nf)
    col_circ = {k: nf + n for n, k in enumerate(S.circ)}
    nu = nf + len(S.circ)
    box = ring_to_nodes(nx, ny, ring)
    ih2 = 1.0 / (h * h)
    rows, cols, vals = [], [], []
    f = np.zeros(nu)
    fj, fi = np.nonzero(fluid_in)
    pid = idx[fj, fi]
    f[pid] = omega[fj - 1, fi - 1]
    rows.append(pid); cols.append(pid); vals.append(np.full(nf, 4.0 * ih2))
    minus_nodes, Gpsi, Gbc, _ = S.ghosts
    mrow = {node: r for r, node in enumerate(minus_nodes)}
    psibar_fixed = np.asarray(psibar_fixed, dtype=np.float64)
    extra_r, extra_c, extra_v = [], [], []
    for di, dj in ex.DIRS:
        qi, qj = fi + di, fj + dj
        isbox = (qi == 0) | (qi == nx) | (qj == 0) | (qj == ny)
        f[pid[isbox]] += box[qj[isbox], qi[isbox]] * ih2
        isfl = ~isbox & ~solid[qj, qi]
        rows.append(pid[isfl]); cols.append(idx[qj[isfl], qi[isfl]]); vals.append(np.full(isfl.sum(), -ih2))
        for p, a, b in zip(pid[~isbox & solid[qj, qi]], qi[~isbox & solid[qj, qi]], qj[~isbox & solid[qj, qi]]):
            r = mrow[(int(a), int(b))]
            row = Gpsi.getrow(r)
            for c, w in zip(row.indices, row.data):
                extra_r.append(p); extra_c.append(idx[c // nx1, c % nx1]); extra_v.append(-w * ih2)
            rowb = Gbc.getrow(r)
            for c, w in zip(rowb.indices, rowb.data):
                k = int(S.cp_body[c])
                f[p] += w * S.psi_b[c] * ih2
                if k in col_circ:
                    extra_r.append(p); extra_c.append(col_circ[k]); extra_v.append(-w * ih2)
                else:
                    f[p] += w * psibar_fixed[k] * ih2
    if extra_r:
        rows.append(np.array(extra_r)); cols.append(np.array(extra_c)); vals.append(np.array(extra_v))
    for k in S.circ:
        lx, rx, ly, ry = S.prob.regions[k]
        rk = col_circ[k]
        coeff = {}

        def add(i, j, v):
            coeff[(i, j)] = coeff.get((i, j), 0.0) + v
        # -[ sum_j (psi_{rx+1,j}-psi_{rx,j}) + sum_i (psi_{i,ry+1}-psi_{i,ry})
        #    - sum_j (psi_{lx,j}-psi_{lx-1,j}) - sum_i (psi_{i,ly}-psi_{i,ly-1}) ] = Gamma_k
        for j in range(ly, ry + 1):
            add(rx + 1, j, -1.0); add(rx, j, 1.0); add(lx, j, 1.0); add(lx - 1, j, -1.0)
        for i in range(lx, rx + 1):
            add(i, ry + 1, -1.0); add(i, ry, 1.0); add(i, ly, 1.0); add(i, ly - 1, -1.0)
        for (i, j), v in coeff.items():
            if v != 0.0:
                rows.append(np.array([rk])); cols.append(np.array([idx[j, i]])); vals.append(np.array([v * ih2]))
        f[rk] = gamma[k] * ih2
    L = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nu, nu))
    return L, f, idx, col_circ


def solve_unreduced(S: Setup, omega=None, ring=None, gamma=None, psibar=None):
    """psi (node array: fluid values, box data, zero in the solid) and psibar per body."""
    P = S.prob
    omega = P.omega if omega is None else omega
    ring = P.psi_box if ring is None else ring
    psibar = np.zeros(S.nb) if psibar is None else np.asarray(psibar, dtype=np.float64)
    gamma = np.zeros(S.nb) if gamma is None else np.asarray(gamma, dtype=np.float64)
    L, f, idx, col_circ = assemble_unreduced(S, omega, ring, gamma, psibar)
    u = spla.spsolve(L.tocsc(), f)
    psi = ring_to_nodes(S.nx, S.ny, ring)
    m = idx >= 0
    psi[m] = u[idx[m]]
    pb = psibar.copy()
    for k, c in col_circ.items():
        pb[k] = u[c]
    return psi, pb


# ----------------------------------------------------------------------------- Schur form
class SchurOperators:
    """Affected points, the operators A and B and the circulation rows of Sec. 4.2."""

    def __init__(self, S: Setup):
        self.S = S
        geo = S.geo
        nx1 = S.nx + 1
        self.ai, self.aj = geo["aff_i"], geo["aff_j"]     # row-major order
        self.asolid = geo["aff_solid"]
        self.abody = geo["aff_body"]
        self.na = len(self.ai)
        minus_nodes, Gpsi, Gbc, _ = S.ghosts
        mrow = {node: r for r, node in enumerate(minus_nodes)}
        ih2 = 1.0 / (S.h * S.h)
        ra, ca, va = [], [], []
        rb, cb, vb = [], [], []
        for a in range(self.na):
            i, j = int(self.ai[a]), int(self.aj[a])
            for di, dj in ex.DIRS:
                qi, qj = i + di, j + dj
                if S.solid[qj, qi] == S.solid[j, i]:
                    continue
                if self.asolid[a]:
                    # solid p: gamma_p = (1/h^2) sum over fluid neighbours of psi_q
                    ra.append(a); ca.append(qj * nx1 + qi); va.append(ih2)
                else:
                    # fluid p: gamma_p = -(1/h^2) sum over solid neighbours of ghost(q)
                    r = mrow[(qi, qj)]
                    row = Gpsi.getrow(r)
                    for c, w in zip(row.indices, row.data):
                        ra.append(a); ca.append(c); va.append(-w * ih2)
                    rowb = Gbc.getrow(r)
                    for c, w in zip(rowb.indices, rowb.data):
                        rb.append(a); cb.append(c); vb.append(-w * ih2)
        nn = (S.ny + 1) * nx1
        self.A = sp.csr_matrix((va, (ra, ca)), shape=(self.na, nn))
        self.B = sp.csr_matrix((vb, (rb, cb)), shape=(self.na, len(S.psi_b)))
        # B applied to the indicator of body k's control points
        self.B1 = np.stack([self.B @ (S.cp_body == k).astype(np.float64) for k in range(S.nb)], axis=1) \
            if S.nb else np.zeros((self.na, 0))

    def scatter(self, gamma):
        """E_a gamma as an interior array."""
        out = np.zeros((self.S.ny - 1, self.S.nx - 1))
        out[self.aj - 1, self.ai - 1] = gamma
        return out

    def apply_A(self, interior):
        nodes = np.zeros((self.S.ny + 1, self.S.nx + 1))
        nodes[1:-1, 1:-1] = interior
        return self.A @ nodes.ravel()


def gmres_mgs(apply, b, tol, restart, max_iter, x0=None):
    """Restarted GMRES with modified Gram-Schmidt and Givens rotations (Saad & Schultz 1986)."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    while True:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm or it >= max_iter:
            return x, it, beta / bnorm
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for j in range(restart):
            w = apply(V[j])
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k_used = j + 1
            if abs(g[j + 1]) <= tol * bnorm or it >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + V[:k_used].T @ y


def solve_schur(S: Setup, omega=None, ring=None, gamma=None, psibar=None,
                tol=1e-13, restart=60, max_iter=2000, ops=None, outer="dirichlet", plane=None):
    """The paper's algorithm (Sec. 4.2): GMRES on the augmented Schur system, then Eq.
    psirecovery.  Returns (psi node array, psibar, gmres iterations, gmres rel. residual).
    outer = "dirichlet": the rectangular solve is the Dirichlet box (DST-I) with box data
    `ring`; outer = "unbounded": it is the free-space solve (poisson_free), the box ring of the
    result is part of the solution and `ring` is ignored; outer = "symmetric": the same with
    the outflow plane through the right box edge (poisson_free(..., sym=True), Sec. 5.2) and
    `plane` the vorticity on the plane column."""
    P = S.prob
    omega = P.omega if omega is None else omega
    free = outer in ("unbounded", "symmetric")
    sym = outer == "symmetric"
    ring = (np.zeros(2 * (S.nx + S.ny)) if free else P.psi_box) if ring is None else ring
    psibar = np.zeros(S.nb) if psibar is None else np.asarray(psibar, dtype=np.float64)
    gamma = np.zeros(S.nb) if gamma is None else np.asarray(gamma, dtype=np.float64)
    O = SchurOperators(S) if ops is None else ops
    h = S.h
    na, circ = O.na, S.circ

    def solve_rect(f, with_ring):
        """Interior values of the rectangular solve (and the node array in free space); the
        plane sources are data, so they enter with the data (with_ring) only."""
        if free:
            nodes = poisson_free(f, h, sym=sym, plane=plane if with_ring else None)
            return nodes[1:-1, 1:-1], nodes
        return poisson_box(f, h, ring if with_ring else None), None

    u0, _ = solve_rect(omega, True)
    rhs_g = O.apply_A(u0) + O.B @ S.psi_b
    for k in range(S.nb):
        if k not in circ:
            rhs_g = rhs_g + O.B1[:, k] * psibar[k]
    rhs_c = np.array([region_sum(omega, P.regions[k]) - gamma[k] / (h * h) for k in circ])
    bvec = np.concatenate([rhs_g, rhs_c])

    def apply(x):
        g = x[:na]
        y = g + O.apply_A(solve_rect(O.scatter(g), False)[0])
        for n, k in enumerate(circ):
            y = y - O.B1[:, k] * x[na + n]
        c = np.array([g[O.abody == k].sum() for k in circ])
        return np.concatenate([y, c])

    x, iters, rel = gmres_mgs(apply, bvec, tol, restart, max_iter)
    g = x[:na]
    psi_in, nodes = solve_rect(omega - O.scatter(g), True)
    psi = nodes.copy() if free else ring_to_nodes(S.nx, S.ny, ring)
    psi[1:-1, 1:-1] = np.where(S.solid[1:-1, 1:-1], 0.0, psi_in)
    pb = psibar.copy()
    for n, k in enumerate(circ):
        pb[k] = x[na + n]
    return psi, pb, iters, rel


# ----------------------------------------------------------------------------- outputs
def extended_psi(S: Setup, psi_nodes, psibar):
    """psi with fourth-order ghosts at A- using psi_b + psibar_k (Sec. 4.2, velocity recovery)."""
    return ex.extend(psi_nodes, S.prob.phi, S.ghosts, S.bc_values(psibar))


def velocity(S: Setup, psi_nodes, psibar):
    """u = (d_y psi, -d_x psi) by centered differences of the extended psi at fluid interior
    nodes; zero in the solid (Sec. 4.2, end).  Returns interior arrays (ux, uy)."""
    e = extended_psi(S, psi_nodes, psibar)
    h = S.h
    ux = (e[2:, 1:-1] - e[:-2, 1:-1]) / (2.0 * h)
    uy = -(e[1:-1, 2:] - e[1:-1, :-2]) / (2.0 * h)
    fl = ~S.solid[1:-1, 1:-1]
    return np.where(fl, ux, 0.0), np.where(fl, uy, 0.0)


def residual(S: Setup, psi_nodes, psibar, omega=None, ring=None, gamma=None, outer="dirichlet", plane=None):
    """Relative residual ||f - L u|| / ||f|| of the un-reduced system (circulation rows in the
    units of omega).  Evaluated matrix-free; `psi_nodes` must carry the box data.  In free
    space (outer = "unbounded" or "symmetric") the box ring of psi_nodes is part of the solution,
    so the known part f carries no box terms."""
    P = S.prob
    omega = P.omega if omega is None else omega
    if outer in ("unbounded", "symmetric"):
        ring = np.zeros(2 * (S.nx + S.ny))
    else:
        ring = P.psi_box if ring is None else ring
    gamma = np.zeros(S.nb) if gamma is None else np.asarray(gamma, dtype=np.float64)
    h = S.h
    e = extended_psi(S, psi_nodes, psibar)
    fl = ~S.solid[1:-1, 1:-1]
    r = np.where(fl, omega - neg_laplacian_5pt(e, h), 0.0)
    # known part f of the rows: omega + box terms + ghost terms carrying psi_b and fixed psibar
    known_bc = psibar.copy()
    for k in S.circ:
        known_bc[k] = 0.0
    zero = np.zeros_like(psi_nodes)
    box_only = ring_to_nodes(S.nx, S.ny, ring)
    ek = ex.extend(zero, P.phi, S.ghosts, S.psi_b + known_bc[S.cp_body])
    ek[0, :], ek[-1, :], ek[:, 0], ek[:, -1] = box_only[0, :], box_only[-1, :], box_only[:, 0], box_only[:, -1]
    f = np.where(fl, omega - neg_laplacian_5pt(ek, h), 0.0)
    rc = np.array([(gamma[k] - discrete_circulation(psi_nodes, P.regions[k])) / (h * h) for k in S.circ])
    fc = np.array([gamma[k] / (h * h) for k in S.circ])
    if outer in ("unbounded", "symmetric"):
        # the ring equations of the free-space system (ring_residual), in units of omega
        rr = ring_residual(psi_nodes, sym=outer == "symmetric", plane=plane, h=h) / (h * h)
        rc = np.concatenate([rc, rr])
        if outer == "symmetric" and plane is not None:
            fc = np.concatenate([fc, plane_potential(S.nx, S.ny, h, plane) / (h * h)])
    num = np.sqrt((r * r).sum() + (rc * rc).sum())
    den = np.sqrt((f * f).sum() + (fc * fc).sum())
    return num / den
