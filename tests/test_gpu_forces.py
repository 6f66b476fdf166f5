"""Control-volume force and moment (App. C) on the GPU: parity with the oracle's sums on the
library's own solve outputs, and the exact Couette flow around a fixed cylinder (zero force,
moment 4 pi nu A R^2) reached at second order through the whole path (IIM solve, velocity,
control-volume kernel)."""
import math

import numpy as np
import pytest
import torch

import paper_2109_13628_gb300 as iim
from oracle import forces as of
from oracle import poisson as op
from paper_2109_13628_gb300 import inputs
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

A, R, C, NU = 0.7, 0.5, (0.03, -0.02), 0.01


def couette_problem(n):
    g = inputs.square_grid(n)
    X, Y = g.nodes()
    phi = inputs.phi_circle(X, Y, C[0], C[1], R)
    r = np.hypot(X - C[0], Y - C[1])
    psi = -A * (0.5 * r * r - R * R * np.log(np.maximum(r, 1e-300)))
    psi_w = -A * (0.5 * R * R - R * R * math.log(R))
    w = np.where(phi >= 0, 2.0 * A, 0.0)
    P = inputs.Problem(grid=g, phi=phi, regions=[inputs.region_around(g, phi)], modes=[0], omega=w[1:-1, 1:-1],
                       psi_box=inputs.box_ring(g, psi), psi_b_fn=lambda x, y, b: np.full_like(x, psi_w),
                       psibar=np.zeros(1), gamma=None, exact=None)
    return P, psi_w


@pytest.mark.parametrize("prec", [iim.IIM_FP64, iim.IIM_MIXED])
def test_cv_terms_match_oracle_and_couette_moment(prec):
    errs = []
    for n in (64, 128, 256):
        P, psi_w = couette_problem(n)
        geo = gu.setup(P)
        out = gu.solve(P, geo, prec=prec, rtol=1e-12, velocity=True)
        box = tuple(int(round(f * n)) for f in (0.2, 0.7, 0.25, 0.8))
        psi_d, ux_d, uy_d = gu.T(out["psi"].ravel()), gu.T(out["ux"].ravel()), gu.T(out["uy"].ravel())
        om_d = gu.T(P.omega.ravel())
        t = iim.iim_cv_terms(geo, psi_d, ux_d, uy_d, om_d, psi_w, box, NU, C)
        # the oracle's sums on the same fields (node arrays with zero box values; the box keeps
        # clear of the grid box)
        nodes = lambda a: np.pad(a, 1)
        solid = P.phi < 0
        ref = of.cv_terms(nodes(out["ux"]), nodes(out["uy"]), nodes(P.omega), nodes(out["psi"]), solid, psi_w,
                          P.grid.h, P.grid.x0, P.grid.y0, box, NU, C)
        assert np.abs(t - ref).max() < 1e-12 * max(1.0, np.abs(ref).max()), (t, ref)
        M = 4 * math.pi * NU * A * R * R
        errs.append(max(abs(t[8] - M), abs(t[4]), abs(t[5])) / M)
        geo.close()
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert errs[-1] < 2e-3 and min(rates) > 1.7, (errs, rates)


def test_cv_box_must_clear_the_body():
    P, psi_w = couette_problem(64)
    geo = gu.setup(P)
    out = gu.solve(P, geo, rtol=1e-12, velocity=True)
    d = [gu.T(out[k].ravel()) for k in ("psi", "ux", "uy")] + [gu.T(P.omega.ravel())]
    with pytest.raises(iim.IIMError) as e:
        iim.iim_cv_terms(geo, *d, psi_w, (30, 40, 30, 40), NU, C)     # cuts through the cylinder
    assert e.value.status == iim.IIM_ERR_BAD_REGION
    with pytest.raises(iim.IIMError):
        iim.iim_cv_terms(geo, *d, psi_w, (1, 40, 10, 50), NU, C)      # edge on the grid box
    geo.close()
