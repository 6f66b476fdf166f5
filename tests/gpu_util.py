"""Helpers of the GPU parity tests: run a Problem through the C ABI."""
import numpy as np
import torch

import paper_2109_13628_gb300 as iim


def dev():
    return torch.device("cuda", 0)


def T(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=dev())


def grid_of(P):
    g = P.grid
    return iim.make_grid(g.x0, g.x1, g.y0, g.y1, g.nx, g.ny)


def setup(P):
    return iim.iim_setup_geometry(grid_of(P), T(P.phi), P.regions, P.modes)


def psi_b_for(P, geo):
    cp = iim.iim_geometry_control_points(geo)
    return P.psi_b_fn(cp["x"].cpu().numpy(), cp["y"].cpu().numpy(), cp["body"].cpu().numpy())


def solve(P, geo, gamma=None, psibar=None, prec=iim.IIM_FP64, rtol=1e-12, velocity=False, guess=None, restart=64,
          max_iter=3000, inner_rtol=0.0, check=True, omega=None):
    g = P.grid
    NXY = (g.nx - 1) * (g.ny - 1)
    psi = torch.empty(NXY, dtype=torch.float64, device=dev())
    ux = torch.empty_like(psi) if velocity else None
    uy = torch.empty_like(psi) if velocity else None
    pb = T(np.zeros(len(P.regions)) if psibar is None else psibar)
    gm = None if gamma is None else T(gamma)
    opts = iim.default_opts(prec=prec, rtol=rtol, restart=restart, max_iter=max_iter,
                            guess=0 if guess is None else 1, inner_rtol=inner_rtol)
    st = iim.iim_poisson_solve(geo, T(P.omega if omega is None else omega), T(psi_b_for(P, geo)), T(P.psi_box), gm, pb,
                               psi, ux, uy, None if guess is None else T(guess), opts=opts, check=check)
    sh = (g.ny - 1, g.nx - 1)
    out = {"psi": psi.cpu().numpy().reshape(sh), "psibar": pb.cpu().numpy(), "stats": st}
    if velocity:
        out["ux"] = ux.cpu().numpy().reshape(sh)
        out["uy"] = uy.cpu().numpy().reshape(sh)
    return out


def nodes_from_interior(P, interior):
    """Node array with the box data of P and the given interior values."""
    from oracle import poisson as op
    g = P.grid
    out = op.ring_to_nodes(g.nx, g.ny, P.psi_box)
    out[1:-1, 1:-1] = interior
    return out


def solve_opts(P, geo, gamma=None, psibar=None, opts=None, velocity=False):
    """Solve with explicit iim_opts (e.g. the preconditioned form)."""
    g = P.grid
    NXY = (g.nx - 1) * (g.ny - 1)
    psi = torch.empty(NXY, dtype=torch.float64, device=dev())
    ux = torch.empty_like(psi) if velocity else None
    uy = torch.empty_like(psi) if velocity else None
    pb = T(np.zeros(len(P.regions)) if psibar is None else psibar)
    gm = None if gamma is None else T(gamma)
    st = iim.iim_poisson_solve(geo, T(P.omega), T(psi_b_for(P, geo)), T(P.psi_box), gm, pb, psi, ux, uy, None,
                               opts=opts)
    sh = (g.ny - 1, g.nx - 1)
    out = {"psi": psi.cpu().numpy().reshape(sh), "psibar": pb.cpu().numpy(), "stats": st}
    if velocity:
        out["ux"] = ux.cpu().numpy().reshape(sh)
        out["uy"] = uy.cpu().numpy().reshape(sh)
    return out
