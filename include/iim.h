/*
 * iim.h -- C ABI of the GB300 immersed interface Poisson library.
 *
 * The library solves the IIM-corrected discrete Poisson problem that reconstructs the
 * streamfunction (and velocity) from vorticity around several immersed bodies, as stated in
 * Gabbard, Gillis, Chatelain & van Rees, "An immersed interface method for the 2D
 * vorticity-velocity Navier-Stokes equations with multiple bodies", Sec. 4.2 (the discrete
 * problem: Eqs. discretepoisson, poissoncorrections, schur, psirecovery, and the augmented
 * system with the circulation rows), with the geometry of Sec. 2.2 / App. A and the
 * polynomial extrapolation of Sec. 2.1.
 *
 * Conventions shared by every entry point
 *   - Grid: the box [x0,x1] x [y0,y1] is split into nx x ny square cells, h = (x1-x0)/nx =
 *     (y1-y0)/ny.  nx and ny must be powers of two in [16, 2048].  Node (i, j) sits at
 *     (x0 + i h, y0 + j h), i = 0..nx, j = 0..ny.  Unknowns live on the interior nodes.
 *   - Layouts (row-major, x fastest, FP64 unless stated otherwise):
 *       node arrays      (ny+1) x (nx+1), element (i, j) at j*(nx+1) + i
 *       interior arrays  (ny-1) x (nx-1), element (i, j) at (j-1)*(nx-1) + (i-1)
 *       box ring         2(nx+ny) values: bottom row j=0 (i=0..nx), top row j=ny (i=0..nx),
 *                        left column i=0 (j=1..ny-1), right column i=nx (j=1..ny-1)
 *   - Level set: phi < 0 is solid, phi >= 0 is fluid (a zero counts as fluid).
 *   - Every array argument is a DEVICE pointer unless marked "host".  All device memory
 *     passed in is owned by the caller; the library owns only what an iim_geometry
 *     allocates (released by iim_destroy_geometry).
 *   - Work is issued on `stream` (NULL = the legacy default stream).  Entry points that
 *     return statistics synchronize that stream before returning.
 *   - Every entry point returns an iim_status; no C++ exception crosses the ABI.
 */
#ifndef IIM_H
#define IIM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* iim_stream; /* identical to cudaStream_t */
typedef struct iim_geometry_s* iim_geometry;
typedef int iim_status;

enum {
    IIM_OK = 0,
    IIM_ERR_INVALID_ARG = -1,   /* null pointer, bad size, grid not a power of two, ... */
    IIM_ERR_UNDERRESOLVED = -2, /* an A- point has no usable extrapolation direction (Sec. 2.2) */
    IIM_ERR_BAD_REGION = -3,    /* an affected point lies in no / several R_k, a region's faces
                                   are not in plain fluid, a body is within 5 nodes of the box,
                                   or a box node is solid */
    IIM_ERR_NONFINITE = -4,     /* NaN/Inf met in the inputs or in a residual */
    IIM_ERR_NOT_CONVERGED = -5, /* iteration caps reached; the best iterate is still written */
    IIM_ERR_TIMEOUT = -6,       /* a bounded device-side wait ran out */
    IIM_ERR_CUDA = -7           /* a CUDA runtime call failed (allocation, launch, ...) */
};

typedef struct { double x0, x1, y0, y1; int nx, ny; } iim_grid;

/* Bounding region R_k of body k: the inclusive box of interior nodes lx..rx, ly..ry (global
 * node indices).  It must contain every affected point of body k and none of another body,
 * and its four boundary faces (Eq. sum_dR_def) must pass between plain fluid nodes. */
typedef struct { int lx, rx, ly, ry; } iim_region;

enum { IIM_BODY_FIXED = 0,       /* psibar_k given (Eq. psibc) */
       IIM_BODY_CIRCULATION = 1  /* Gamma_k given, psibar_k solved for (Eq. discretecircconstraint) */ };

enum { IIM_FP64 = 0,   /* every step in FP64: the plain iteration */
       IIM_MIXED = 1   /* FP32 rectangular solves inside FP64 iterative refinement of the
                          un-reduced residual; FP64 extrapolation weights, residual, Krylov
                          inner products and circulation rows */ };

typedef struct {
    int prec;          /* IIM_FP64 or IIM_MIXED */
    double rtol;       /* target: relative residual ||f - L u||_2 / ||f||_2 of the un-reduced
                          FP64 system (fluid rows + circulation rows / h^2) */
    int max_iter;      /* cap on Krylov iterations summed over refinements */
    int restart;       /* GMRES restart length, 1..64 */
    int max_refine;    /* cap on outer refinement steps */
    int guess;         /* 0: start from psi = 0; 1: psi_guess is the first iterate (kept only if it
                          lowers the un-reduced residual); 2: psi_guess seeds the Krylov unknowns
                          of the first correction: the body constants psibar0_k it implies
                          (quadratic extrapolation of psi_guess to the crossings, averaged per
                          body) and x0 = c [A psi_guess + B sum_k psibar0_k 1_k ; psibar0] with
                          the c that minimises ||b - S x0||, so ||b - S x0|| <= ||b||; dropped
                          when c = 0 -- the learned-guess path */
    double inner_rtol; /* Krylov tolerance of each correction solve (<= 0: library default,
                          rtol/20 in FP64 mode, 1e-4 in mixed mode) */
    int precond;       /* 0: plain GMRES; 1: right-precondition GMRES with the dense inverse of
                          the Schur matrix (built on first use, see iim_build_preconditioner);
                          2: each correction applies that inverse once, x = M b, with no Krylov
                          iterations; when a correction fails to halve the FP64 residual the
                          remaining corrections use mode 1 (stats fallback bit 1);
                          3: mode 1 with the inner Krylov operator S applied as the dense FP32
                          matrix formed with the inverse (one matrix-vector product instead of
                          three transform passes and a gather per iteration); the transforms
                          remain for each correction's right-hand side and recovery, and the
                          FP64 residual of the un-reduced system still decides convergence.
                          Falls back to mode 1 when 4 (|A| + circulation bodies) floats exceed
                          200 KB */
} iim_opts;

typedef struct {
    int iters;           /* Krylov iterations, all refinements */
    int refinements;     /* correction solves performed */
    int fallback;        /* bit 0: a caller guess raised the residual and was dropped; bit 1:
                            direct corrections (precond 2) handed over to GMRES */
    int status;          /* same value as returned */
    double rel_res;      /* final un-reduced FP64 relative residual */
    double gmres_rel_res;/* last Krylov relative residual */
    double circ_err_max; /* max_k |Gamma_k - (-h sum_dRk grad_h psi . n)| over circulation bodies */
    float ms;            /* wall time of the call on the stream (CUDA events) */
    double seed_rel_res; /* guess = 2: ||b - S x0|| / ||b|| of the seed of the first correction
                            (1 without a seed) */
    int iters_first;     /* Krylov iterations of the first correction (the one a seed starts) */
} iim_stats;

/* Geometry setup (Sec. 2.2, App. A): finds the control points (grid-line crossings of the
 * zero level set, located by a cubic fit of four level-set samples, Newton and deflation),
 * the affected points A+ / A-, the fourth-order ghost stencils (Sec. 2.1) and the per-body
 * labels (from R_k), and allocates the solver's device workspace.
 *   grid       host; nx, ny powers of two in [16, 2048]
 *   phi_nodes  node array (device, FP64)
 *   n_bodies   number of bodies, 0..64; regions, modes: host arrays of that length
 * Errors: IIM_ERR_INVALID_ARG, IIM_ERR_BAD_REGION, IIM_ERR_UNDERRESOLVED, IIM_ERR_CUDA.
 * On error *out is NULL and nothing stays allocated.  Synchronizes `stream`. */
iim_status iim_setup_geometry(const iim_grid* grid, const double* phi_nodes, int n_bodies,
                              const iim_region* regions, const int* modes, iim_stream stream,
                              iim_geometry* out);

/* Sizes of the geometry: control points |C|, affected points |A|, bodies.  Host outputs,
 * any may be NULL. */
iim_status iim_geometry_info(iim_geometry g, int* n_control, int* n_affected, int* n_bodies);

/* Control points in canonical order (x-edges by (j, i), then y-edges by (j, i)): position,
 * owning body, edge axis (0 = x, 1 = y), the edge's lower node (i, j) and t = distance from
 * the fluid node to the crossing in units of h.  Device outputs of length |C|, any NULL. */
iim_status iim_geometry_control_points(iim_geometry g, double* x, double* y, int* body, int* axis,
                                       int* edge_i, int* edge_j, double* t, iim_stream stream);

/* Affected points in row-major node order: node (i, j), solid flag (1 = A-), body.
 * Device outputs of length |A|, any NULL. */
iim_status iim_geometry_affected_points(iim_geometry g, int* node_i, int* node_j, int* solid,
                                        int* body, iim_stream stream);

/* IIM Poisson solve (Sec. 4.2 and the full-algorithm step "Velocity Reconstruction",
 * Sec. 5.5): finds psi with -nabla_h^2 psi_ext = omega at every fluid interior node, psi =
 * psi_b + psibar_k on body k, box data psi_box, and -h sum_{dR_k} (grad_h psi).n = Gamma_k for
 * circulation-mode bodies; then u = (d_y psi, -d_x psi) by centered differences of the
 * fourth-order extension of psi (Sec. 4.2, end).
 *   omega      interior array; values at solid nodes are ignored
 *   psi_b      |C| values at the control points (canonical order)
 *   psi_box    box ring, or NULL for zero box data
 *   gamma      n_bodies values (entries of fixed-mode bodies ignored), or NULL for zeros
 *   psibar     n_bodies values: read for fixed bodies, written for circulation bodies
 *              (ignored and may be NULL on a geometry in Neumann mode, iim_geometry_set_wall_condition)
 *   psi_out    interior array: fluid values, 0 in the solid
 *   ux_out, uy_out  interior arrays (0 in the solid), or NULL to skip the velocity
 *   psi_guess  interior array used when opts->guess is 1 or 2, else ignored (may be NULL)
 *   opts       host; NULL = FP64, rtol 1e-10, restart 40, max_iter 2000, max_refine 8
 *   stats      host, may be NULL
 * From the second solve on a geometry (no guess, precond 0 or 1, no profiling), the whole solve
 * -- refinements, GMRES cycles and iterations -- runs as one CUDA graph whose loops are decided
 * on the device; it is captured again when the arguments or the geometry's tile settings change.
 * Refinement stops when the relative residual is <= rtol.  With circulation bodies the solve
 * then makes the circulation constraint exact to rounding by capacitance: the first solve on
 * a geometry also computes, once, the response to unit circulation of each circulation body
 * (one solve each, kept with the geometry), and every solve adds the combination of them that
 * cancels Gamma_k - (-h sum_dRk grad_h psi . n).
 * Errors: IIM_ERR_INVALID_ARG, IIM_ERR_NONFINITE, IIM_ERR_NOT_CONVERGED (outputs still hold
 * the best iterate), IIM_ERR_CUDA.  Synchronizes `stream` (convergence tests read one scalar
 * per Krylov iteration).  Not re-entrant on one geometry: calls that share an iim_geometry
 * must be serialized, since they share its workspace. */
iim_status iim_poisson_solve(iim_geometry g, const double* omega, const double* psi_b,
                             const double* psi_box, const double* gamma, double* psibar,
                             double* psi_out, double* ux_out, double* uy_out,
                             const double* psi_guess, const iim_opts* opts, iim_stats* stats,
                             iim_stream stream);

/* Many independent IIM Poisson solves in flight at once (batched workloads of mixed grid sizes
 * and geometries).  Problem k uses geoms[k] (all distinct: each geometry owns the workspace
 * of its solve) and the k-th pointer of every array argument, with the meaning of
 * iim_poisson_solve; psi_box, gamma, ux_out, uy_out may be NULL arrays (then NULL for every
 * problem).  The problems go to n_streams streams, largest first.  A problem whose geometry
 * has already been solved once runs as one whole-solve graph launch (see iim_poisson_solve),
 * all of them launched from the calling thread without waiting; first solves (host-driven, with
 * their set-up) are shared by n_streams worker threads.  The work is ordered after prior work
 * on `stream` and `stream` waits for all of it; the call returns when every problem is done.
 * stats: host, n entries or NULL.
 * Returns the first non-OK status of any problem (all problems are attempted).  The paper
 * solves one problem at a time; batching is this library's throughput mode. */
iim_status iim_poisson_solve_batched(int n, iim_geometry const* geoms, const double* const* omega,
                                     const double* const* psi_b, const double* const* psi_box,
                                     const double* const* gamma, double* const* psibar,
                                     double* const* psi_out, double* const* ux_out, double* const* uy_out,
                                     const iim_opts* opts, iim_stats* stats, int n_streams,
                                     iim_stream stream);

/* How iim_poisson_solve_batched and iim_poisson_solve_batched_host run problems that have been
 * solved once already, with iim_opts.precond 1 or 3 and no guess.  max_group >= 2 (default 4):
 * the problems of equal grid size (and equal iim_geometry_set_tiles / _set_lines settings) are
 * split into groups of at most max_group problems (sizes as even as possible), and each group
 * advances in lockstep -- one kernel launch per step of the solve for every problem of the
 * group, the refinement, cycle and iteration loops continuing on the device while any problem of
 * the group needs them (one CUDA graph per group); the groups run concurrently on their own
 * streams.  max_group 0 or 1: one whole-solve graph per problem on the call's streams.  Each
 * problem's results, iteration and refinement counts are bitwise the same either way (the same
 * arithmetic in the same order per problem).  Larger groups mean fewer launches and wider
 * kernels; more groups mean more overlap of the small latency-bound Krylov kernels of one group
 * with the transforms of another.  Process-wide; returns the previous setting.  No counterpart
 * in the paper, which solves one problem at a time. */
int iim_set_lockstep(int max_group);

/* iim_poisson_solve_batched on HOST buffers: every array argument (omega, psi_b, psi_box,
 * gamma, psibar in/out, psi_out, ux_out, uy_out) is host memory, preferably page-locked so
 * that the copies run asynchronously.  Each problem's inputs are copied to device staging
 * arrays kept with its geometry (allocated on the first such call), solved, and its outputs
 * copied back, all on the problem's stream, so the copies of some problems overlap the solves
 * of others.  When a problem's psi_out (and ux_out, uy_out if given) are page-locked host
 * memory the device can address at the same pointer (cudaHostAlloc / cudaHostRegister under
 * unified addressing), the solve's last kernel writes them there directly instead (no staging
 * or copy).  Returns when every output is in host memory.  Same errors as
 * iim_poisson_solve_batched. */
iim_status iim_poisson_solve_batched_host(int n, iim_geometry const* geoms, const double* const* omega,
                                          const double* const* psi_b, const double* const* psi_box,
                                          const double* const* gamma, double* const* psibar,
                                          double* const* psi_out, double* const* ux_out,
                                          double* const* uy_out, const iim_opts* opts, iim_stats* stats,
                                          int n_streams, iim_stream stream);

/* Tile width of the column pass of the geometry's rectangular solves: 2, 4 or 8 columns per
 * block (FP32 transforms use 4 or 8, FP64 transforms 2 or 4; the nearest supported width is
 * taken).  Chosen per grid size by the autotuner of the Python package.  Errors:
 * IIM_ERR_INVALID_ARG. */
iim_status iim_geometry_set_tiles(iim_geometry g, int cols_per_block);

/* Exterior condition of the geometry's solves (Sec. 4.1: bounded and unbounded domains;
 * Sec. 4.2: the rectangular solution operator nabla_h^-2 with those conditions; Sec. 5.2:
 * outflow boundaries).
 *   outer 0 (default): Dirichlet box -- psi_box is the data on the box ring, gauge psibar_0 = 0.
 *   outer 1: unbounded -- psi is the free-space solution on the infinite lattice: the solution
 *     operator is the convolution psi(x) = h^2 sum_y G(x - y) f(y) with the lattice Green's
 *     function G of the five-point Laplacian in the gauge G(0, 0) = 0 (the paper leaves the
 *     gauge to the free constant of the Green's function), evaluated exactly (to
 *     rounding) by James's method: one box solve of the source, the ring sum of G against the
 *     box solve next to the box, and one box solve of the ring values.  psi_box is ignored: the
 *     box ring of psi is part of the solution (iim_geometry_outer_ring); omega must vanish outside
 *     the box.  psi is the perturbation field: for a free stream u_inf add u_inf x x (lattice-
 *     harmonic, so give psi_b minus it at the control points).  guess mode 1 is refused.
 *   outer 2: unbounded with an outflow plane through the right box edge (node column nx): the
 *     vorticity is mirrored evenly across that plane (Sec. 5.2), so psi is the free-space field
 *     of omega, of its images (2 nx - i, j) and of the vorticity on the plane column itself
 *     (iim_geometry_set_plane_vorticity; zero until set), which is its own image:
 *     psi(x) = h^2 { sum_y [G(x - y) + G(x - y*)] omega(y) + sum_j G(x - (nx, j)) w_j }; psi is
 *     even about the plane (u_y = 0 and d u_x / dx = 0 there).  The same method with the ring
 *     kernel G(x - y) + G(x* - y); the G table covers 2 nx columns.
 * Changing it drops the geometry's preconditioner, circulation responses and solve graphs (they
 * are rebuilt by the next solve).  The first switch to 1 or 2 for a grid size builds that
 * size's G table (device, shared, kept until exit; synchronizes the device).
 * Errors: IIM_ERR_INVALID_ARG (outer not 0, 1 or 2), IIM_ERR_CUDA. */
iim_status iim_geometry_set_outer(iim_geometry g, int outer);

/* With the outflow plane (outer 2): the vorticity on the plane column, w (NY = ny - 1 values,
 * rows j = 1..ny-1, host or device memory), copied into the geometry (stream-ordered) and used
 * by every later solve until set again; the circulation responses leave it out.  Errors:
 * IIM_ERR_INVALID_ARG (null pointer, or the geometry is not in mode 2), IIM_ERR_CUDA. */
iim_status iim_geometry_set_plane_vorticity(iim_geometry g, const double* w, iim_stream stream);

/* In free space (outer 1): psi on the box ring of the last solve (device, 2 (nx + ny) values in
 * the ring layout).  Asynchronous.  Errors: IIM_ERR_INVALID_ARG (not in free space). */
iim_status iim_geometry_outer_ring(iim_geometry g, double* ring, iim_stream stream);

/* How the column pass of the geometry's rectangular solves (FP32 and FP64) works.  After the
 * row transforms, every x mode turns the 5-point operator along a column into a tridiagonal
 * system (the FFT / tridiagonal form of the Sec. 4.2 rectangular solve).  1 (default) solves
 * these systems directly: the two Thomas recurrences as segmented scans, with the elimination
 * factors tabulated through their complements 1 - e_j; O(ny) work per column.  0 uses the
 * column DST pair with the eigenvalue division.  Both compute the same discrete inverse to
 * rounding.  Changing it drops the dense preconditioner and the circulation responses (rebuilt
 * by the next solve that uses them, with the new pass).  Errors: IIM_ERR_INVALID_ARG (mode not
 * 0 or 1). */
iim_status iim_geometry_set_column_solver(iim_geometry g, int mode);

/* Wall condition of the geometry's ghost stencils (Sec. 2.1).  0 (default): Dirichlet, the
 * ghost at an A- node g along a usable direction d is the cubic through the crossing (carrying
 * psi_b + psibar_k) and the fluid nodes g+2d, g+3d, g+4d, at g.  1: Neumann, the variant of
 * Sec. 2.1 for a derivative condition: the cubic p through the same three fluid nodes whose
 * derivative along the line at the crossing is the wall datum, at g; the ghost is again the
 * mean over usable directions.  In Neumann mode the psi_b argument of the solves is that datum,
 * d . grad u at each control point with d the unit grid direction from the solid node of the
 * control point's edge to its fluid node (into the fluid); there are no body constants: the
 * psibar arguments are ignored (read as zeros, never written; NULL is accepted).  This is the
 * solve of the total-pressure problem of Sec. 5.4 (iim_total_pressure).  Requires every body in
 * IIM_BODY_FIXED mode for kind 1.  The transport and vorticity-boundary kernels do not use these
 * stencils (they keep their own Dirichlet extensions).  Changing it rewrites the stencils
 * (synchronizes `stream`) and drops the preconditioner, circulation responses and solve graphs.
 * Errors: IIM_ERR_INVALID_ARG (kind not 0 or 1, or kind 1 with a circulation body), IIM_ERR_CUDA. */
iim_status iim_geometry_set_wall_condition(iim_geometry g, int kind, iim_stream stream);

/* Threads per transformed line for 1024-point lines: 32 (default: one warp, fewest
 * instructions, best when many solves share the GPU) or 64 (two warps per line: lower latency
 * of one solve, about 6 % more instructions).  Other line lengths use one warp.  Errors:
 * IIM_ERR_INVALID_ARG. */
iim_status iim_geometry_set_lines(iim_geometry g, int threads_per_line);

/* Builds the dense Schur-complement preconditioner of a geometry: the matrix S of the augmented
 * system of Sec. 4.2 (gamma plus circulation unknowns), one column per FP32 operator
 * application, and its inverse by Gauss-Jordan elimination with partial pivoting in FP32,
 * kept as an (ns x 2ns) FP32 array on the device (ns = |A| + circulation bodies).  The paper
 * solves with plain GMRes; this is a one-time cost per geometry that pays when many solves
 * share the geometry (time stepping).  Its milliseconds go to *setup_ms (host, may be NULL).
 * Errors: IIM_ERR_NOT_CONVERGED (singular pivot), IIM_ERR_CUDA.  Synchronizes `stream`. */
iim_status iim_build_preconditioner(iim_geometry g, float* setup_ms, iim_stream stream);

/* Rectangular Dirichlet-box solve u = -nabla_h^{-2} f (Sec. 4.2: the FFT solution operator,
 * here a 2D DST-I for the Dirichlet box): -nabla_h^2 u = f on the interior nodes with box data.
 *   f, u       interior arrays (may alias)
 *   psi_box    box ring or NULL (zero)
 *   prec       IIM_FP64 (transforms in FP64) or IIM_MIXED (transforms in FP32)
 *   work       caller workspace of 2 (nx-1)(ny-1) doubles
 * Errors: IIM_ERR_INVALID_ARG, IIM_ERR_CUDA.  Asynchronous on `stream`. */
iim_status iim_box_poisson(const iim_grid* grid, const double* f, const double* psi_box,
                           double* u, int prec, double* work, iim_stream stream);

/* Pass timing of the rectangular solve (no counterpart in the paper: a measurement hook for
 * benchmarks, not part of any solve).  Runs, in precision `prec` (IIM_FP64 or IIM_MIXED = FP32
 * transforms) and with the geometry's current column pass and tile width, the three passes of
 * the Sec. 4.2 rectangular solve on `batch` synthetic fields of g's grid: forward row transforms
 * of dense FP64 fields, the column pass and the inverse row transforms, each pass one launch
 * over all fields; each pass is launched `reps` times back to back inside a CUDA
 * graph of its own, timed with CUDA events around one launch of that graph.  Outputs (host): us[3] = average device time per
 * launch in microseconds, bytes[3] = algorithmic bytes one launch moves (inputs read once,
 * outputs written once).  The call allocates and frees its own device scratch (3 fields), uses
 * a stream of its own and returns after the measurement.  Errors: IIM_ERR_INVALID_ARG (null
 * pointers, batch or reps < 1, bad prec), IIM_ERR_CUDA. */
iim_status iim_time_box_passes(iim_geometry g, int prec, int batch, int reps, double* us, double* bytes);

/* Allocation-free variant of iim_box_poisson.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- code running while a CUDA graph is
 * being captured (where cudaMalloc would break the capture), real-time loops and embedded or
 * foreign-language hosts that must not touch the device allocator, and applications whose
 * memory pool already owns all free device memory.  Same arguments and results as
 * iim_box_poisson without `work`: the scratch is a static device array of the library of
 * 1024 * 1026 doubles (8.4 MB), held by every GPU that loads the library until the process
 * exits.  Limits: nx, ny <= 1024 (larger grids return IIM_ERR_INVALID_ARG and a message in
 * iim_last_error_message).  The first call on a device performs a one-time set-up on that
 * device (twiddle tables, the scratch address, kernel attributes); make that first call
 * before any stream capture.  Afterwards calls allocate nothing on the device or the host;
 * every call shares the one scratch array, so calls that overlap on the GPU (different
 * streams, or other threads) race -- serialize them.  The per-kernel profiler
 * (iim_profile_begin) records events with allocation; keep it off around this call.
 * Errors: IIM_ERR_INVALID_ARG, IIM_ERR_CUDA.  Asynchronous on `stream`. */
iim_status iim_box_poisson_noalloc(const iim_grid* grid, const double* f, const double* psi_box, double* u,
                                   int prec, iim_stream stream);

/* Control-volume force and moment on a stationary body (App. C: the momentum formulation of
 * Noca, Eq. Fm with its tensor gamma, and the moment formulation of Eqs. Mm1 and Mm2), density 1.
 * The control volume is the node box `box` (global node indices lx..rx, ly..ry; 2 <= lx < rx <=
 * nx - 2, likewise in y) minus the body inside it; the box edges and their neighbours must be
 * plain fluid (else IIM_ERR_BAD_REGION).  Surface integrals use the trapezoidal rule on the box's
 * node lines and centred differences.
 *   psi, ux, uy  interior arrays of a solve (psi 0 in the solid, as iim_poisson_solve writes it)
 *   omega        interior array of the vorticity
 *   psi_wall     psi on the body's wall (psi_b + psibar_k; constant on a stationary no-slip wall)
 *   nu           viscosity;  xbar  host, the moment centre
 *   out          host, 9 values: A_x, A_y, B_x, B_y, C_x, C_y, P, Q, R with
 *                A = int_V u, B = oint x cross (n cross u), C = oint n . gamma,
 *                P = int_V x cross u, Q = oint |x|^2/2 (n cross u), R = oint lambda(n),
 *                so that F = -dA/dt - dB/dt + C and M = -dP/dt + dQ/dt + R (x from xbar); the
 *                time derivatives come from a series of calls (the volume integrals are
 *                evaluated through psi: A = (oint psi n_y, -oint psi n_x),
 *                P = -oint psi (x.n) + 2 int_box psi~, psi~ = psi_wall in the body).
 * Synchronizes `stream`.  Errors: IIM_ERR_INVALID_ARG, IIM_ERR_BAD_REGION, IIM_ERR_CUDA. */
iim_status iim_cv_terms(iim_geometry g, const double* psi, const double* ux, const double* uy, const double* omega,
                        double psi_wall, const iim_region* box, double nu, const double xbar[2], double* out,
                        iim_stream stream);

/* Conservative vorticity transport right-hand side with the IIM boundary treatment (Sec. 3:
 * Eqs. upwind, 2dshuconserve, Sec. 3.2) and the Kelvin ODE (Sec. 5.1, Eq. discreteKelvinChoice)
 * for a given velocity; omega_b from the velocity by the local vorticity boundary condition of
 * Sec. 5.3 (its stencil figure is missing from the paper; the library's reading is a
 * three-node quadratic along the grid line and a one-sided second-order difference across it
 * that uses u_b).
 *   omega, ux, uy  interior arrays (values at solid nodes ignored)
 *   u_b            2 |C| values: u_x at the control points, then u_y (NULL: no-slip, zero)
 *   Uinf           host, 2 values: velocity at and beyond the box
 *   nu             viscosity (>= 0)
 *   omega_b_in     |C| values of a prescribed wall vorticity, or NULL to derive omega_b from
 *                  the velocity (Sec. 5.3)
 *   omega_b_out    |C| values or NULL (the omega_b used)
 *   rhs_out        interior array: d omega / dt (0 in the solid)
 *   dgamma_out     n_bodies values: -h sum_{dR_k}(f + q).n, or NULL
 * Box: vorticity 0 at and beyond the box except the right edge (outflow), which copies the
 * last interior column.  Errors: IIM_ERR_INVALID_ARG, IIM_ERR_CUDA.  Asynchronous. */
iim_status iim_transport_rhs(iim_geometry g, const double* omega, const double* ux, const double* uy,
                             const double* u_b, const double Uinf[2], double nu, const double* omega_b_in,
                             double* omega_b_out, double* rhs_out, double* dgamma_out, iim_stream stream);

/* The data of the total-pressure problem (Sec. 5.4) from a flow: H = (p - p_inf) +
 * (|u|^2 - |u_inf|^2) / 2 solves nabla^2 H = div(u x omega k) (Eq. pressurepoisson) with a
 * Neumann wall condition (Eq. totalpressurebc).
 *   f_out      interior array: f = -div(u x omega k) = -(d_x(u_y omega) - d_y(u_x omega)) at fluid
 *              nodes (the right-hand side of -nabla_h^2 H = f), centred differences of the
 *              products; at A- nodes the third-order extensions (u with u_b, omega with omega_b),
 *              at and beyond the box the box values of iim_transport_rhs (u = Uinf; omega 0,
 *              copied from the last interior column at the right edge); 0 in the solid
 *   data_out   |C| values: the wall datum of the Neumann stencils (iim_geometry_set_wall_condition),
 *              d . grad H at each crossing.  On a stationary no-slip wall grad(|u|^2/2) =
 *              (grad u)^T u vanishes and Eq. pressuregrad1 gives grad H = grad p = nu k x grad omega:
 *              the normal part is Eq. totalpressurebc's -nu d omega/ds, the tangential part the nu
 *              d omega/dn of Eq. pressureflux.  An x-line needs d_y omega, a y-line d_x omega at the
 *              crossing: the cross-line stencil of the vorticity boundary condition (Sec. 5.3, as
 *              in iim_transport_rhs) on the vorticity extended at third order with omega_b.
 *   other arguments as in iim_transport_rhs (u_b only extends the velocity: the wall relation
 *              above assumes a stationary wall).
 * Errors: IIM_ERR_INVALID_ARG, IIM_ERR_CUDA.  Asynchronous. */
iim_status iim_total_pressure_problem(iim_geometry g, const double* omega, const double* ux, const double* uy,
                                      const double* u_b, const double Uinf[2], double nu, const double* omega_b_in,
                                      double* omega_b_out, double* f_out, double* data_out, iim_stream stream);

/* A field (interior array, fluid values) at every control point (|C| outputs, canonical
 * order): the quadratic through the fluid node next to the crossing and the next two fluid
 * interior nodes along its grid line, evaluated at the crossing (a third-order extrapolation,
 * Sec. 5.4's surface pressure), the line or the node value where those nodes are not fluid.
 * Errors: IIM_ERR_INVALID_ARG.  Asynchronous. */
iim_status iim_wall_values(iim_geometry g, const double* field, double* out, iim_stream stream);

/* The global surface-pressure method of Sec. 5.4 on a geometry in Neumann mode: the problem data
 * of iim_total_pressure_problem (stationary no-slip walls, omega_b from the velocity), the IIM
 * solve of -nabla_h^2 H = f with the Neumann stencils (iim_poisson_solve: opts, stats and
 * errors as there; H_box is the box ring of H or NULL for zero, ignored in free space), and the
 * surface values of H (iim_wall_values) into H_wall_out (|C| values, or NULL).  The static
 * pressure on the wall is p - p_inf = H + |u_inf|^2 / 2.  The right-hand side and the datum are
 * kept in the geometry's own scratch.  Errors: IIM_ERR_INVALID_ARG (also when the geometry is
 * not in Neumann mode), those of iim_poisson_solve.  Synchronizes `stream`. */
iim_status iim_total_pressure(iim_geometry g, const double* omega, const double* ux, const double* uy,
                              const double Uinf[2], double nu, const double* H_box, double* H_out,
                              double* H_wall_out, const iim_opts* opts, iim_stats* stats, iim_stream stream);

/* One time step of the full algorithm (Sec. 5.5): three stages of the low-storage RK3 of
 * Williamson (1980) (A = 0, -5/9, -153/128; B = 1/3, 15/16, 8/15) on (omega, Gamma_k); each stage
 * reconstructs psi and u with iim_poisson_solve (Gamma as given), evaluates omega_b, the
 * transport right-hand side and the Kelvin ODE, then updates.
 *   omega          interior array, in/out (kept 0 in the solid)
 *   gamma          n_bodies, in/out (device)
 *   psibar         n_bodies, in/out (device): fixed values / last solved values
 *   u_b            2 |C| values (u_x then u_y) or NULL (no-slip)
 *   psi_b          |C| values or NULL (zero)
 *   psi_box        box ring or NULL (zero)
 *   Uinf, nu       as in iim_transport_rhs
 *   c_stab, dt_inout  host: if *dt_inout <= 0 the step is c_stab times the stable step of the
 *                  RK3 polygon (App. B): 1/dt_max = max(|u_x|+|u_y|)/(1.620 h) + nu/(0.314 h^2),
 *                  from the velocity of the first stage; the step used is written back
 *   opts           Poisson solve options (NULL: defaults of iim_poisson_solve)
 *   per_stage      host, 3 entries or NULL
 * Errors: those of iim_poisson_solve, IIM_ERR_INVALID_ARG.  Synchronizes `stream`. */
iim_status iim_rk3_step(iim_geometry g, double* omega, double* gamma, double* psibar, const double* u_b,
                        const double* psi_b, const double* psi_box, const double Uinf[2], double nu,
                        double c_stab, double* dt_inout, const iim_opts* opts, iim_stats* per_stage,
                        iim_stream stream);

/* iim_rk3_step with a wall velocity that changes during the step, as for a body whose rotation
 * rate follows a prescribed law (the Navier-Stokes convergence study of Sec. 6.1 drives the
 * cylinder's wall with the Lamb-Oseen velocity at the current time).  Stage st (0, 1, 2) of the
 * Williamson scheme sits at time t + c_st dt, c = (0, 1/3, 3/4), and uses
 *   u_b + c_st dt u_b_rate.
 *   u_b_rate       2 |C| values (du_b/dt, u_x then u_y), device; required
 * Everything else as iim_rk3_step (u_b NULL = zero at the start of the step).  A wall velocity
 * linear in time over one step keeps the scheme third order in time.
 * Errors: those of iim_rk3_step; IIM_ERR_INVALID_ARG when u_b_rate is NULL. */
iim_status iim_rk3_step_moving_wall(iim_geometry g, double* omega, double* gamma, double* psibar,
                                    const double* u_b, const double* u_b_rate, const double* psi_b,
                                    const double* psi_box, const double Uinf[2], double nu, double c_stab,
                                    double* dt_inout, const iim_opts* opts, iim_stats* per_stage,
                                    iim_stream stream);

/* ---- Learned initial guess (no counterpart in the paper).  A fully convolutional network of
 * 3x3 dilated convolutions (zero padding, ReLU between layers, BF16 weights, FP32 accumulation)
 * maps per-pixel inputs to one output channel; trained with a masked mean-squared error and
 * Adam by the library's own forward/backward kernels.  Tensors are device FP32 arrays of shape
 * (batch, channels, height, width), row-major.  The solver judges every guess by its residual
 * (iim_opts.guess = 1 falls back to zero when the guess raises it). */
typedef struct iim_net_s* iim_net;

/* Layers l = 0..n_layers-1: in_channels -> hidden -> ... -> hidden -> 1, dilation dilations[l]
 * (host array); He-uniform weights from `seed`, zero biases.  in_channels, hidden <= 32. */
iim_status iim_net_create(int in_channels, int hidden, int n_layers, const int* dilations,
                          unsigned long long seed, iim_net* out);
long long iim_net_num_params(iim_net net);
/* FP32 parameters (host), per layer the weights (out, in, 3, 3) then the biases.  Setting them
 * also resets the Adam state.  Errors: IIM_ERR_INVALID_ARG (size), IIM_ERR_CUDA. */
iim_status iim_net_get_params(iim_net net, float* host, long long n);
iim_status iim_net_set_params(iim_net net, const float* host, long long n);
/* y (batch, 1, h, w) = net(x (batch, in_channels, h, w)).  Asynchronous. */
iim_status iim_net_forward(iim_net net, int batch, int height, int width, const float* x, float* y,
                           iim_stream stream);
/* Gradient of sum(dy * net(x)) with respect to every parameter, copied to grad_host (host, may
 * be NULL).  Synchronizes `stream` when grad_host is given. */
iim_status iim_net_backward(iim_net net, int batch, int height, int width, const float* x, const float* dy,
                            float* grad_host, iim_stream stream);
/* One Adam step (beta 0.9 / 0.999) on loss = sum(mask (net(x) - target)^2) / sum(mask); mask
 * may be NULL (all ones); the loss before the step goes to *loss (host, may be NULL; then the
 * call is asynchronous). */
iim_status iim_net_train_step(iim_net net, int batch, int height, int width, const float* x,
                              const float* target, const float* mask, float lr, float* loss,
                              iim_stream stream);
/* Network input for a solve on an (nx x ny)-cell grid: three planes of the interior grid,
 * omega * s_omega (0 in the solid), phi * s_phi (level set at the interior nodes of the node
 * array phi_nodes) and u_box * s_box (the rectangular solve of omega, iim_box_poisson). */
iim_status iim_net_prepare_input(int nx, int ny, const double* omega, const double* phi_nodes,
                                 const double* u_box, float s_omega, float s_phi, float s_box, float* x,
                                 iim_stream stream);
/* psi_guess = u_box + y / s_out (n values). */
iim_status iim_net_compose_guess(long long n, const double* u_box, const float* y, float s_out,
                                 double* psi_guess, iim_stream stream);
/* Convolutions on the tensor cores: on = 2 (the default) every layer, 1 the hidden 32 -> 32
 * layers only, 0 none (the CUDA-core kernel).  A convolution on the tensor cores (forward, and the
 * input gradient of training) is an implicit GEMM on the fifth-generation tensor cores: the layer
 * input is rounded to BF16, the products with the BF16 weights are summed in FP32 in tensor
 * memory; layers with fewer than 16 or 32 channels are padded with zero channels to the MMA
 * shape.  The weight gradient stays on the CUDA cores.  Layers off the tensor cores keep FP32
 * inputs.  Errors: IIM_ERR_INVALID_ARG (net NULL, on not 0, 1 or 2). */
iim_status iim_net_set_tensor_cores(iim_net net, int on);
/* *on = the current setting; *timed_out = 1 if a tensor-core convolution of this net ever gave up
 * waiting (one second) for its MMAs and skipped its output, else 0.  Synchronizes the device.
 * Errors: IIM_ERR_INVALID_ARG (NULL argument), IIM_ERR_CUDA. */
iim_status iim_net_tensor_core_status(iim_net net, int* on, int* timed_out);
void iim_net_destroy(iim_net net);

/* Number of kernels the library has launched in this process (all threads, all devices);
 * monotonic.  Lets a caller count the launches inside a timed region. */
long long iim_launch_count(void);

/* Opt-in per-kernel timing (instrumentation, not part of the method): between
 * iim_profile_begin and iim_profile_end, every kernel the calling thread launches is bracketed
 * by CUDA events on its stream.  iim_profile_end waits for those events and writes one record
 * per kernel name (launch count, summed milliseconds, summed algorithmic bytes and flops) into
 * `out` (host, `capacity` entries; the names are static strings) and returns the number of
 * distinct names (which may exceed `capacity`). */
typedef struct { const char* name; long long launches; double ms; double bytes; double flops; } iim_kernel_stat;
iim_status iim_profile_begin(void);
int iim_profile_end(iim_kernel_stat* out, int capacity);

/* Text of the last CUDA failure recorded by this thread (empty when none). */
const char* iim_last_error_message(void);

/* Releases everything the geometry allocated.  NULL is ignored. */
void iim_destroy_geometry(iim_geometry g);

/* Static, human-readable name of a status code. */
const char* iim_status_string(iim_status s);

#ifdef __cplusplus
}
#endif
#endif /* IIM_H */
