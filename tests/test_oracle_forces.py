"""Pins of the oracle's control-volume force and moment (App. C, Eqs. Fm, Mm1, Mm2) on an exact
steady Navier-Stokes flow around a stationary no-slip cylinder: u_theta = A (r - R^2 / r) (the
Couette flow outside a fixed cylinder; vorticity 2A everywhere in the fluid).  By symmetry the
force is zero; the wall shear nu (du/dr - u/r) = 2 nu A gives the moment 4 pi nu A R^2.  The
control-volume formulas hold for any box around the body, so boxes off centre are used too."""
import math

import numpy as np
import pytest

from oracle import forces as of


def couette_nodes(n, A=0.7, R=0.5, c=(0.03, -0.02), half=2.0):
    h = 2 * half / n
    x = -half + h * np.arange(n + 1)
    X, Y = np.meshgrid(x, x)
    dx, dy = X - c[0], Y - c[1]
    r = np.hypot(dx, dy)
    solid = r < R
    ut = np.where(solid, 0.0, A * (r - R * R / np.maximum(r, 1e-300)))
    u = np.where(solid, 0.0, -ut * dy / np.maximum(r, 1e-300))
    v = np.where(solid, 0.0, ut * dx / np.maximum(r, 1e-300))
    w = np.where(solid, 0.0, 2 * A)
    psi = np.where(solid, 0.0, -A * (0.5 * r * r - R * R * np.log(np.maximum(r, 1e-300))))
    psi_w = -A * (0.5 * R * R - R * R * math.log(R))
    return h, -half, u, v, w, psi, solid, psi_w


@pytest.mark.parametrize("box_frac", [(0.3, 0.7, 0.25, 0.75), (0.2, 0.65, 0.3, 0.8)])
def test_couette_moment_and_zero_force_second_order(box_frac):
    A, R, c, nu = 0.7, 0.5, (0.03, -0.02), 0.01
    errs = []
    for n in (64, 128, 256):
        h, x0, u, v, w, psi, solid, psi_w = couette_nodes(n, A, R, c)
        box = tuple(int(round(f * n)) for f in box_frac)
        t = of.cv_terms(u, v, w, psi, solid, psi_w, h, x0, x0, box, nu, c)
        M_exact = 4 * math.pi * nu * A * R * R
        errs.append(max(abs(t[8] - M_exact) / M_exact, abs(t[4]) / M_exact, abs(t[5]) / M_exact))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert errs[-1] < 1e-3 and min(rates) > 1.8, (errs, rates)


def test_couette_volume_integrals():
    """A = int_V u and P = int_V x cross u (box centred on the cylinder, half width L):
    A = 0 by symmetry, P = A [8 L^4 / 3 - 4 L^2 R^2 + pi R^4 / 2]; second order."""
    Acoef, R, nu = 0.7, 0.5, 0.01
    errs = []
    for n in (64, 128, 256):
        h, x0, u, v, w, psi, solid, psi_w = couette_nodes(n, Acoef, R, (0.0, 0.0))
        m = n // 2
        k = n // 4
        box = (m - k, m + k, m - k, m + k)
        L = k * h
        t = of.cv_terms(u, v, w, psi, solid, psi_w, h, x0, x0, box, nu, (0.0, 0.0))
        P_exact = Acoef * (8 * L ** 4 / 3 - 4 * L * L * R * R + math.pi * R ** 4 / 2)
        errs.append(max(abs(t[0]), abs(t[1]), abs(t[6] - P_exact)) / abs(P_exact))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert errs[-1] < 1e-3 and min(rates) > 1.8, (errs, rates)


def test_force_moment_time_difference():
    """force_moment applies F = -dA/dt - dB/dt + C and M = -dP/dt + dQ/dt + R with a central
    difference: exact for terms linear in time."""
    a = np.arange(9.0)
    s = [a, a + 0.5 * np.arange(1, 10), a + 1.0 * np.arange(1, 10)]
    F, M = of.force_moment(s, 0.5)
    d = np.arange(1, 10) * 1.0
    assert np.allclose(F, -d[0:2] - d[2:4] + s[1][4:6]) and np.isclose(M, -d[6] + d[7] + s[1][8])
