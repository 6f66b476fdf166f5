"""Plain, slow FP64 CPU oracle for the immersed interface Poisson hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never imports, links or calls it,
and this package imports nothing from the product path; the two share only the seeded
input generators in ``paper_2109_13628_gb300/inputs.py`` (which hold no method arithmetic).

Every function restates the paper (Gabbard, Gillis, Chatelain, van Rees, "An immersed
interface method for the 2D vorticity-velocity Navier-Stokes equations with multiple
bodies") and cites the section or equation it follows.  Library primitives used as steps:
numpy/scipy dense and sparse linear algebra, scipy's DST-I.

Modules
  geometry       App. A control points, Sec. 2.2 affected sets, body labels from R_k
  extrapolation  Sec. 2.1 polynomial extrapolation, Sec. 2.2 averaging / nonconvex fallback
  poisson        Sec. 4.2: 5-point Laplacian, Dirichlet-box DST-I solver, the un-reduced IIM
                 system (the definition of the discrete result), the Schur-complement GMRES
                 form, circulation, velocity, residual
  transport      Sec. 3, Sec. 5.1, 5.3, 5.5, App. B: vorticity BC, conservative transport
                 RHS, Kelvin ODE, low-storage RK3, stable time step
  lgf            Sec. 4.1 / 4.2: lattice Green's function of the five-point Laplacian (the
                 free-space rectangular solve)
  forces         App. C: control-volume force and moment
  net            the learned initial guess's convolution network, its loss and gradients
  pressure       Sec. 5.4: total-pressure Poisson problem -- right-hand side, Neumann wall
                 datum, the IIM solve with the Neumann extrapolation (Sec. 2.1), surface values

Parity status: every function is pinned by a test in tests/test_oracle_*.py.  The vorticity
boundary condition stencils (Sec. 5.3) are a reading of a figure missing from the paper; they
are pinned by what the paper does fix -- that they are second order: exact for quadratic
velocity fields, and second-order convergent at every control point when fed the exact
Lamb-Oseen velocity around the Sec. 6.1 cylinder.
"""
