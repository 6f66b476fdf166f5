"""Lattice Green's function of the five-point Laplacian: the kernel of the free-space
rectangular solve (Sec. 4.1: unbounded domains, psi from a convolution of the source with a
Green's function whose arbitrary constant fixes the gauge; Sec. 4.2: the FFT solution
operator nabla_h^-2 with unbounded boundary conditions).

Test infrastructure: imported only by the tests, the smoke check and the benchmark's CPU legs.

G is the solution on the integer lattice Z^2 of -L G = delta, with L the five-point stencil
(sum of the four neighbours minus four times the centre), growing like -(1/2 pi) log r, in the
gauge G(0, 0) = 0.  From the Fourier representation of L^-1,
    -G(m, n) = (1 / (2 pi)^2) int int (1 - cos(m t + n s)) / (4 - 2 cos t - 2 cos s) dt ds,
and the s-integral done in closed form (1/2pi) int cos(n s) / (b - 2 cos s) ds = e^(-|n| a) / (2
sinh a) with cosh a = 2 - cos t, b = 4 - 2 cos t:
    -G(m, n) = (1 / 2 pi) int_0^pi (1 - cos(m t) e^(-|n| a(t))) / sinh a(t) dt,
an integrand that is analytic on [0, pi] (the singularities of numerator and denominator at
t = 0 cancel).  On the grid of spacing h the free-space solution of -nabla_h^2 psi = f is
psi(x) = h^2 sum_y G(x - y) f(y).

Pinned (tests/test_oracle_free.py) by what the mathematics fixes: G(1, 0) = -1/4 (from the
equation at the origin and the lattice symmetry), G(1, 1) = -1/pi (a classical closed form),
-L G = delta at every tested point, the far field -(1/2 pi)(log r + euler_gamma + (3/2) log 2)
+ O(r^-2), and the composite rule against scipy's adaptive quadrature.
"""
from __future__ import annotations

import functools

import numpy as np
from scipy import integrate


def _integrand(t, m, n):
    """(1 - cos(m t) e^(-n a)) / sinh a with cosh a = 2 - cos t, written without cancellation:
    1 - cos(m t) e^(-n a) = 2 sin^2(m t / 2) - cos(m t) (e^(-n a) - 1)."""
    a = np.arccosh(2.0 - np.cos(t))
    num = 2.0 * np.sin(0.5 * m * t) ** 2 - np.cos(m * t) * np.expm1(-n * a)
    return num / np.sinh(a)


def lgf_quad(m: int, n: int) -> float:
    """G(m, n) by scipy's adaptive quadrature (small |m|, |n|)."""
    m, n = abs(int(m)), abs(int(n))
    if m == 0 and n == 0:
        return 0.0
    v, _ = integrate.quad(lambda t: _integrand(t, m, n), 0.0, np.pi, limit=400, epsabs=1e-15, epsrel=1e-13)
    return -v / (2.0 * np.pi)


@functools.lru_cache(maxsize=8)
def _gauss_panels(panels: int, order: int = 16):
    x, w = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(0.0, np.pi, panels + 1)
    mid, half = 0.5 * (edges[1:] + edges[:-1]), 0.5 * (edges[1:] - edges[:-1])
    t = (mid[:, None] + half[:, None] * x[None, :]).ravel()
    wt = (half[:, None] * w[None, :]).ravel()
    return t, wt


@functools.lru_cache(maxsize=8)
def lgf_table(M: int, N: int) -> np.ndarray:
    """G(m, n) for 0 <= m <= M, 0 <= n <= N as an (N + 1, M + 1) array [n, m], by a composite
    16-point Gauss-Legendre rule on uniform panels of [0, pi] (at least 4 panels per period of
    cos(m t) and per e-fold of e^(-n a)).  Read-only (cached)."""
    K = max(M, N, 1)
    panels = max(64, 4 * K)
    t, wt = _gauss_panels(panels)
    a = np.arccosh(2.0 - np.cos(t))
    sh = np.sinh(a)
    m = np.arange(M + 1)[:, None]
    out = np.empty((N + 1, M + 1))
    s2 = 2.0 * np.sin(0.5 * m * t[None, :]) ** 2
    cm = np.cos(m * t[None, :])
    for n in range(N + 1):
        num = s2 - cm * np.expm1(-n * a)[None, :]
        out[n, :] = -(num / sh[None, :]) @ wt / (2.0 * np.pi)
    out[0, 0] = 0.0
    out.setflags(write=False)
    return out


def lgf_full(nx: int, ny: int) -> np.ndarray:
    """K[a, b] = G(a - ny, b - nx) for the offsets of an (ny + 1) x (nx + 1) node array."""
    G = lgf_table(nx, ny)
    iy = np.abs(np.arange(-ny, ny + 1))
    ix = np.abs(np.arange(-nx, nx + 1))
    return G[iy[:, None], ix[None, :]]
