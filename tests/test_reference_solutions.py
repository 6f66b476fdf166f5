"""Pins of the closed-form flows the Navier-Stokes GPU tests compare against: the Lamb-Oseen
vortex (Sec. 4.3 / 6.1) and the impulsively rotated cylinder (Sec. 6.2, App. D).  Each is
checked against mathematics it must satisfy, not against a retyping of itself."""
import math

import numpy as np
import pytest

from paper_2109_13628_gb300 import inputs


def test_lamb_oseen_streamfunction_velocity_and_rate():
    """u = (d psi/dy, -d psi/dx), -Laplacian psi = omega and d u/dt, by centred differences."""
    c = inputs.LAMB_OSEEN_CYLINDER
    x = np.linspace(0.3, 0.7, 41)
    X, Y = np.meshgrid(x, x)
    X, Y = X + 1e-3, Y - 2e-3
    e = 1e-4
    args = (c["xc"], c["yc"], c["gamma"])
    nt = c["nu"] * 1.3
    psi = lambda a, b: inputs.psi_lamb_oseen(a, b, *args, nt)
    w, ux, uy = inputs.lamb_oseen(X, Y, *args, nt)
    assert np.abs((psi(X, Y + e) - psi(X, Y - e)) / (2 * e) - ux).max() < 2e-5
    assert np.abs(-(psi(X + e, Y) - psi(X - e, Y)) / (2 * e) - uy).max() < 2e-5
    lap = (psi(X + e, Y) + psi(X - e, Y) + psi(X, Y + e) + psi(X, Y - e) - 4 * psi(X, Y)) / e ** 2
    assert np.abs(-lap - w).max() < 1e-4 * np.abs(w).max()
    t, dt = 1.3, 1e-5
    _, a1, b1 = inputs.lamb_oseen(X, Y, *args, c["nu"] * (t + dt))
    _, a0, b0 = inputs.lamb_oseen(X, Y, *args, c["nu"] * (t - dt))
    rx, ry = inputs.lamb_oseen_rate(X, Y, *args, c["nu"], t)
    assert np.abs((a1 - a0) / (2 * dt) - rx).max() < 1e-7
    assert np.abs((b1 - b0) / (2 * dt) - ry).max() < 1e-7


def test_rotated_cylinder_closed_forms():
    """No slip at the wall; fluid at rest away from it at small t; the plane-wall (Stokes
    first problem) limits u = erfc(d / 2 sqrt(t)) and omega_wall sqrt(pi t) -> -1 as t -> 0;
    vorticity = (1/r) d(r u)/dr; u -> 1/r (the potential vortex) as t grows."""
    pytest.importorskip("scipy")
    for t in (1e-3, 0.02, 0.3):
        assert abs(inputs.rotated_cylinder_velocity(1.0, t) - 1.0) < 1e-12
    assert abs(inputs.rotated_cylinder_velocity(2.0, 1e-3)) < 1e-10
    t = 1e-5
    for d in (0.002, 0.006):
        assert abs(inputs.rotated_cylinder_velocity(1.0 + d, t) - math.erfc(d / (2 * math.sqrt(t)))) < 5e-3
    assert abs(inputs.rotated_cylinder_vorticity(1.0, t) * math.sqrt(math.pi * t) + 1.0) < 5e-3
    for r, t in ((1.0, 0.01), (1.3, 0.02), (1.8, 0.2)):
        e = 1e-4
        d = ((r + e) * inputs.rotated_cylinder_velocity(r + e, t)
             - (r - e) * inputs.rotated_cylinder_velocity(r - e, t)) / (2 * e) / r
        if r == 1.0:   # one-sided at the wall
            d = ((r + 2 * e) * inputs.rotated_cylinder_velocity(r + 2 * e, t) * -1
                 + 4 * (r + e) * inputs.rotated_cylinder_velocity(r + e, t) - 3 * r) / (2 * e) / r
        assert abs(d - inputs.rotated_cylinder_vorticity(r, t)) < 1e-5 * max(1.0, abs(d))
    assert abs(inputs.rotated_cylinder_velocity(1.5, 1e4) - 1 / 1.5) < 0.02
