"""Thin ctypes binding of libiim.so: the same entry points as include/iim.h, with torch CUDA
tensors marshalled to device pointers and the current torch stream passed through.  Every
step of the computation runs in the library's CUDA kernels; there is no CPU fallback, and a
missing library raises."""
from __future__ import annotations

import ctypes
import os

import numpy as np

import torch

from . import build as _build

IIM_OK = 0
IIM_ERR_INVALID_ARG = -1
IIM_ERR_UNDERRESOLVED = -2
IIM_ERR_BAD_REGION = -3
IIM_ERR_NONFINITE = -4
IIM_ERR_NOT_CONVERGED = -5
IIM_ERR_TIMEOUT = -6
IIM_ERR_CUDA = -7
IIM_BODY_FIXED, IIM_BODY_CIRCULATION = 0, 1
IIM_FP64, IIM_MIXED = 0, 1

# (name, restype, argtypes) of every function declared in include/iim.h
_vp, _i, _d, _ip = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int)


class iim_grid(ctypes.Structure):
    _fields_ = [("x0", _d), ("x1", _d), ("y0", _d), ("y1", _d), ("nx", _i), ("ny", _i)]


class iim_region(ctypes.Structure):
    _fields_ = [("lx", _i), ("rx", _i), ("ly", _i), ("ry", _i)]


class iim_opts(ctypes.Structure):
    _fields_ = [("prec", _i), ("rtol", _d), ("max_iter", _i), ("restart", _i), ("max_refine", _i),
                ("guess", _i), ("inner_rtol", _d), ("precond", _i)]


class iim_stats(ctypes.Structure):
    _fields_ = [("iters", _i), ("refinements", _i), ("fallback", _i), ("status", _i), ("rel_res", _d),
                ("gmres_rel_res", _d), ("circ_err_max", _d), ("ms", ctypes.c_float), ("seed_rel_res", _d),
                ("iters_first", _i)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class iim_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong), ("ms", _d), ("bytes", _d), ("flops", _d)]


SIGNATURES = [
    ("iim_setup_geometry", _i, [ctypes.POINTER(iim_grid), _vp, _i, ctypes.POINTER(iim_region), _ip, _vp,
                                ctypes.POINTER(_vp)]),
    ("iim_geometry_info", _i, [_vp, _ip, _ip, _ip]),
    ("iim_geometry_control_points", _i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("iim_geometry_affected_points", _i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("iim_poisson_solve", _i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(iim_opts),
                               ctypes.POINTER(iim_stats), _vp]),
    ("iim_box_poisson", _i, [ctypes.POINTER(iim_grid), _vp, _vp, _vp, _i, _vp, _vp]),
    ("iim_box_poisson_noalloc", _i, [ctypes.POINTER(iim_grid), _vp, _vp, _vp, _i, _vp]),
    ("iim_build_preconditioner", _i, [_vp, ctypes.POINTER(ctypes.c_float), _vp]),
    ("iim_poisson_solve_batched", _i, [_i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(iim_opts),
                                       _vp, _i, _vp]),
    ("iim_poisson_solve_batched_host", _i, [_i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                            ctypes.POINTER(iim_opts), _vp, _i, _vp]),
    ("iim_geometry_set_tiles", _i, [_vp, _i]),
    ("iim_geometry_set_lines", _i, [_vp, _i]),
    ("iim_geometry_set_column_solver", _i, [_vp, _i]),
    ("iim_time_box_passes", _i, [_vp, _i, _i, _i, ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    ("iim_geometry_set_plane_vorticity", _i, [_vp, _vp, _vp]),
    ("iim_geometry_set_outer", _i, [_vp, _i]),
    ("iim_geometry_outer_ring", _i, [_vp, _vp, _vp]),
    ("iim_cv_terms", _i, [_vp, _vp, _vp, _vp, _vp, _d, ctypes.POINTER(iim_region), _d, ctypes.POINTER(_d), _vp, _vp]),
    ("iim_net_create", _i, [_i, _i, _i, _ip, ctypes.c_ulonglong, ctypes.POINTER(_vp)]),
    ("iim_net_num_params", ctypes.c_longlong, [_vp]),
    ("iim_net_get_params", _i, [_vp, _vp, ctypes.c_longlong]),
    ("iim_net_set_params", _i, [_vp, _vp, ctypes.c_longlong]),
    ("iim_net_forward", _i, [_vp, _i, _i, _i, _vp, _vp, _vp]),
    ("iim_net_backward", _i, [_vp, _i, _i, _i, _vp, _vp, _vp, _vp]),
    ("iim_net_train_step", _i, [_vp, _i, _i, _i, _vp, _vp, _vp, ctypes.c_float, ctypes.POINTER(ctypes.c_float), _vp]),
    ("iim_net_prepare_input", _i, [_i, _i, _vp, _vp, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp, _vp]),
    ("iim_net_compose_guess", _i, [ctypes.c_longlong, _vp, _vp, ctypes.c_float, _vp, _vp]),
    ("iim_net_set_tensor_cores", _i, [_vp, _i]),
    ("iim_net_tensor_core_status", _i, [_vp, _ip, _ip]),
    ("iim_net_destroy", None, [_vp]),
    ("iim_transport_rhs", _i, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_d), _d, _vp, _vp, _vp, _vp, _vp]),
    ("iim_geometry_set_wall_condition", _i, [_vp, _i, _vp]),
    ("iim_total_pressure_problem", _i, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_d), _d, _vp, _vp, _vp, _vp, _vp]),
    ("iim_wall_values", _i, [_vp, _vp, _vp, _vp]),
    ("iim_total_pressure", _i, [_vp, _vp, _vp, _vp, ctypes.POINTER(_d), _d, _vp, _vp, _vp, ctypes.POINTER(iim_opts),
                                ctypes.POINTER(iim_stats), _vp]),
    ("iim_rk3_step", _i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_d), _d, _d, ctypes.POINTER(_d),
                          ctypes.POINTER(iim_opts), ctypes.POINTER(iim_stats), _vp]),
    ("iim_rk3_step_moving_wall", _i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_d), _d, _d,
                                      ctypes.POINTER(_d), ctypes.POINTER(iim_opts), ctypes.POINTER(iim_stats), _vp]),
    ("iim_last_error_message", ctypes.c_char_p, []),
    ("iim_launch_count", ctypes.c_longlong, []),
    ("iim_set_lockstep", _i, [_i]),
    ("iim_profile_begin", _i, []),
    ("iim_profile_end", _i, [ctypes.POINTER(iim_kernel_stat), _i]),
    ("iim_destroy_geometry", None, [_vp]),
    ("iim_status_string", ctypes.c_char_p, [_i]),
]

_lib = None


def library_path() -> str:
    return _build.OUT


def load(build_if_missing: bool = True):
    """Loads libiim.so (building it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libiim.so not found at {path}; run paper_2109_13628_gb300/build.py")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class IIMError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.iim_status_string(status).decode()
        extra = lib.iim_last_error_message().decode()
        super().__init__(f"{where}: {msg}" + (f" ({extra})" if extra and status == IIM_ERR_CUDA else ""))
        self.status = status


def _check(st, where):
    if st != IIM_OK:
        raise IIMError(st, where)


def _ptr(t, dtype=None, numel=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def make_grid(x0, x1, y0, y1, nx, ny):
    return iim_grid(float(x0), float(x1), float(y0), float(y1), int(nx), int(ny))


class Geometry:
    """Owns an iim_geometry handle (released by iim_destroy_geometry)."""

    def __init__(self, handle, grid, n_bodies, modes):
        self.handle = handle
        self.grid = grid
        self.n_bodies = n_bodies
        self.modes = list(modes)
        nc, na, nb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().iim_geometry_info(handle, nc, na, nb), "iim_geometry_info")
        self.n_control, self.n_affected = nc.value, na.value

    def close(self):
        if self.handle:
            load().iim_destroy_geometry(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def iim_setup_geometry(grid: iim_grid, phi_nodes: torch.Tensor, regions, modes, stream=None) -> Geometry:
    lib = load()
    nb = len(regions)
    R = (iim_region * max(nb, 1))(*[iim_region(*map(int, r)) for r in regions])
    M = (ctypes.c_int * max(nb, 1))(*[int(m) for m in modes])
    out = ctypes.c_void_p()
    st = lib.iim_setup_geometry(ctypes.byref(grid), _ptr(phi_nodes, torch.float64, (grid.nx + 1) * (grid.ny + 1), "phi"),
                                nb, R, M, _stream(stream), ctypes.byref(out))
    _check(st, "iim_setup_geometry")
    return Geometry(out, grid, nb, modes)


def iim_geometry_info(g: Geometry):
    return g.n_control, g.n_affected, g.n_bodies


def iim_geometry_control_points(g: Geometry, stream=None):
    n = g.n_control
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {k: torch.empty(n, dtype=torch.float64, device=dev) for k in ("x", "y", "t")}
    out.update({k: torch.empty(n, dtype=torch.int32, device=dev) for k in ("body", "axis", "i", "j")})
    st = load().iim_geometry_control_points(g.handle, _ptr(out["x"]), _ptr(out["y"]), _ptr(out["body"]), _ptr(out["axis"]),
                                            _ptr(out["i"]), _ptr(out["j"]), _ptr(out["t"]), _stream(stream))
    _check(st, "iim_geometry_control_points")
    return out


def iim_geometry_affected_points(g: Geometry, stream=None):
    n = g.n_affected
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {k: torch.empty(n, dtype=torch.int32, device=dev) for k in ("i", "j", "solid", "body")}
    st = load().iim_geometry_affected_points(g.handle, _ptr(out["i"]), _ptr(out["j"]), _ptr(out["solid"]),
                                             _ptr(out["body"]), _stream(stream))
    _check(st, "iim_geometry_affected_points")
    return out


def default_opts(prec=IIM_FP64, rtol=1e-10, max_iter=2000, restart=64, max_refine=12, guess=0, inner_rtol=0.0,
                 precond=0):
    return iim_opts(int(prec), float(rtol), int(max_iter), int(restart), int(max_refine), int(guess), float(inner_rtol),
                    int(precond))


def iim_geometry_set_tiles(g: "Geometry", cols_per_block: int):
    _check(load().iim_geometry_set_tiles(g.handle, int(cols_per_block)), "iim_geometry_set_tiles")


def iim_geometry_set_lines(g: "Geometry", threads_per_line: int):
    """32 (one warp per 1024-point line, the default) or 64 (lower single-solve latency)."""
    _check(load().iim_geometry_set_lines(g.handle, int(threads_per_line)), "iim_geometry_set_lines")


def iim_geometry_set_column_solver(g: "Geometry", mode: int):
    """Column pass of the FP32 rectangular solves: 1 tridiagonal solves per x mode (default),
    0 the column DST pair."""
    _check(load().iim_geometry_set_column_solver(g.handle, int(mode)), "iim_geometry_set_column_solver")


def iim_time_box_passes(g: "Geometry", prec: int, batch: int = 1, reps: int = 20):
    """Device time per launch (us) and algorithmic bytes per launch of the three passes of the
    rectangular solve (forward rows, columns, inverse rows) on `batch` fields (see iim.h)."""
    us, by = (_d * 3)(), (_d * 3)()
    _check(load().iim_time_box_passes(g.handle, int(prec), int(batch), int(reps), us, by), "iim_time_box_passes")
    return {"us": list(us), "bytes": list(by)}


def iim_geometry_set_plane_vorticity(g: "Geometry", w, stream=None):
    """With the outflow plane (outer 2): the vorticity on the plane column (ny - 1 values, a CUDA
    tensor of FP64; see iim.h)."""
    _check(load().iim_geometry_set_plane_vorticity(g.handle, _ptr(w, torch.float64, g.grid.ny - 1, "w"),
                                                   _stream(stream)), "iim_geometry_set_plane_vorticity")


def iim_geometry_set_outer(g: "Geometry", outer: int):
    """Exterior condition: 0 Dirichlet box (default), 1 unbounded (free space), 2 unbounded with
    the outflow plane through the right box edge."""
    _check(load().iim_geometry_set_outer(g.handle, int(outer)), "iim_geometry_set_outer")


def iim_geometry_outer_ring(g: "Geometry", ring=None, stream=None):
    """psi on the box ring of the last free-space solve (device tensor, ring layout)."""
    n = 2 * (g.grid.nx + g.grid.ny)
    if ring is None:
        ring = torch.empty(n, dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
    _check(load().iim_geometry_outer_ring(g.handle, _ptr(ring, torch.float64, n, "ring"), _stream(stream)),
           "iim_geometry_outer_ring")
    return ring


def iim_cv_terms(g: "Geometry", psi, ux, uy, omega, psi_wall, box, nu, xbar, stream=None):
    """Control-volume force / moment quantities (A_x, A_y, B_x, B_y, C_x, C_y, P, Q, R) on the node
    box `box` = (lx, rx, ly, ry) around one stationary body (see iim.h)."""
    nxy = (g.grid.nx - 1) * (g.grid.ny - 1)
    out = (_d * 9)()
    xb = (_d * 2)(*xbar)
    reg = iim_region(*[int(v) for v in box])
    _check(load().iim_cv_terms(g.handle, _ptr(psi, torch.float64, nxy, "psi"), _ptr(ux, torch.float64, nxy, "ux"),
                               _ptr(uy, torch.float64, nxy, "uy"), _ptr(omega, torch.float64, nxy, "omega"),
                               float(psi_wall), ctypes.byref(reg), float(nu), xb, out, _stream(stream)),
           "iim_cv_terms")
    return np.array(out[:])


def _host_ptr(t, dtype=None, numel=None, name="tensor"):
    """Host pointer of a contiguous CPU tensor (or None); page-locked memory lets the copies run
    asynchronously."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a CPU tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _ptr_array(tensors, dtype, sizes, name, host=False):
    """Host array of device pointers (NULL entries allowed) or None when every entry is None."""
    if tensors is None or all(t is None for t in tensors):
        return None
    arr = (_vp * len(tensors))()
    for k, (t, n) in enumerate(zip(tensors, sizes)):
        p = (_host_ptr if host else _ptr)(t, dtype, n, f"{name}[{k}]")
        arr[k] = p.value if p is not None else None
    return arr


def iim_poisson_solve_batched(geoms, omega, psi_b, psi_box, gamma, psibar, psi_out, ux_out=None, uy_out=None,
                              opts: "iim_opts | None" = None, n_streams=8, stream=None, check=True):
    """Solves len(geoms) independent problems concurrently; returns (status, [stats dicts])."""
    n = len(geoms)
    f64 = torch.float64
    nxy = [(g.grid.nx - 1) * (g.grid.ny - 1) for g in geoms]
    G = (_vp * n)(*[g.handle.value if isinstance(g.handle, ctypes.c_void_p) else g.handle for g in geoms])
    stats = (iim_stats * n)()
    o = opts if opts is not None else default_opts()
    none = [None] * n
    st = load().iim_poisson_solve_batched(
        n, G, _ptr_array(omega, f64, nxy, "omega"), _ptr_array(psi_b, f64, [g.n_control for g in geoms], "psi_b"),
        _ptr_array(psi_box or none, f64, [2 * (g.grid.nx + g.grid.ny) for g in geoms], "psi_box"),
        _ptr_array(gamma or none, f64, [g.n_bodies for g in geoms], "gamma"),
        _ptr_array(psibar, f64, [g.n_bodies for g in geoms], "psibar"), _ptr_array(psi_out, f64, nxy, "psi_out"),
        _ptr_array(ux_out or none, f64, nxy, "ux_out"), _ptr_array(uy_out or none, f64, nxy, "uy_out"),
        ctypes.byref(o), stats, int(n_streams), _stream(stream))
    if check:
        _check(st, "iim_poisson_solve_batched")
    return st, [stats[k].as_dict() for k in range(n)]


def iim_poisson_solve_batched_host(geoms, omega, psi_b, psi_box, gamma, psibar, psi_out, ux_out=None, uy_out=None,
                                   opts: "iim_opts | None" = None, n_streams=8, stream=None, check=True):
    """iim_poisson_solve_batched on host (CPU, preferably pinned) tensors: copies in, solves and
    copies out per problem on its stream; returns (status, [stats dicts])."""
    n = len(geoms)
    f64 = torch.float64
    nxy = [(g.grid.nx - 1) * (g.grid.ny - 1) for g in geoms]
    G = (_vp * n)(*[g.handle.value if isinstance(g.handle, ctypes.c_void_p) else g.handle for g in geoms])
    stats = (iim_stats * n)()
    o = opts if opts is not None else default_opts()
    none = [None] * n
    st = load().iim_poisson_solve_batched_host(
        n, G, _ptr_array(omega, f64, nxy, "omega", True),
        _ptr_array(psi_b, f64, [g.n_control for g in geoms], "psi_b", True),
        _ptr_array(psi_box or none, f64, [2 * (g.grid.nx + g.grid.ny) for g in geoms], "psi_box", True),
        _ptr_array(gamma or none, f64, [g.n_bodies for g in geoms], "gamma", True),
        _ptr_array(psibar, f64, [g.n_bodies for g in geoms], "psibar", True),
        _ptr_array(psi_out, f64, nxy, "psi_out", True), _ptr_array(ux_out or none, f64, nxy, "ux_out", True),
        _ptr_array(uy_out or none, f64, nxy, "uy_out", True), ctypes.byref(o), stats, int(n_streams), _stream(stream))
    if check:
        _check(st, "iim_poisson_solve_batched_host")
    return st, [stats[k].as_dict() for k in range(n)]


def iim_build_preconditioner(g: "Geometry", stream=None) -> float:
    """Builds the dense Schur-complement preconditioner; returns its set-up milliseconds."""
    ms = ctypes.c_float()
    _check(load().iim_build_preconditioner(g.handle, ctypes.byref(ms), _stream(stream)), "iim_build_preconditioner")
    return ms.value


def iim_poisson_solve(g: Geometry, omega, psi_b, psi_box, gamma, psibar, psi_out, ux_out=None, uy_out=None,
                      psi_guess=None, opts: iim_opts | None = None, stream=None, check=True):
    """Returns the iim_stats as a dict; raises IIMError on a non-OK status when `check`."""
    lib = load()
    NXY = (g.grid.nx - 1) * (g.grid.ny - 1)
    f64 = torch.float64
    stats = iim_stats()
    o = opts if opts is not None else default_opts()
    st = lib.iim_poisson_solve(g.handle, _ptr(omega, f64, NXY, "omega"), _ptr(psi_b, f64, g.n_control, "psi_b"),
                               _ptr(psi_box, f64, 2 * (g.grid.nx + g.grid.ny), "psi_box"),
                               _ptr(gamma, f64, g.n_bodies, "gamma"), _ptr(psibar, f64, g.n_bodies, "psibar"),
                               _ptr(psi_out, f64, NXY, "psi_out"), _ptr(ux_out, f64, NXY, "ux_out"),
                               _ptr(uy_out, f64, NXY, "uy_out"), _ptr(psi_guess, f64, NXY, "psi_guess"),
                               ctypes.byref(o), ctypes.byref(stats), _stream(stream))
    d = stats.as_dict()
    d["status"] = st
    if check:
        _check(st, "iim_poisson_solve")
    return d


def iim_box_poisson(grid: iim_grid, f, psi_box, u, prec, work, stream=None):
    NXY = (grid.nx - 1) * (grid.ny - 1)
    st = load().iim_box_poisson(ctypes.byref(grid), _ptr(f, torch.float64, NXY, "f"),
                                _ptr(psi_box, torch.float64, 2 * (grid.nx + grid.ny), "psi_box"),
                                _ptr(u, torch.float64, NXY, "u"), int(prec), _ptr(work, torch.float64, None, "work"),
                                _stream(stream))
    _check(st, "iim_box_poisson")


def iim_box_poisson_noalloc(grid: iim_grid, f, psi_box, u, prec, stream=None):
    """iim_box_poisson without a workspace argument: the library's static device scratch is
    used, for callers that cannot allocate device memory (nx, ny <= 1024; calls that overlap
    on the GPU race)."""
    NXY = (grid.nx - 1) * (grid.ny - 1)
    st = load().iim_box_poisson_noalloc(ctypes.byref(grid), _ptr(f, torch.float64, NXY, "f"),
                                        _ptr(psi_box, torch.float64, 2 * (grid.nx + grid.ny), "psi_box"),
                                        _ptr(u, torch.float64, NXY, "u"), int(prec), _stream(stream))
    _check(st, "iim_box_poisson_noalloc")


def iim_status_string(st: int) -> str:
    return load().iim_status_string(st).decode()


def iim_destroy_geometry(g: Geometry):
    g.close()


def iim_launch_count() -> int:
    return int(load().iim_launch_count())


def iim_set_lockstep(max_group: int) -> int:
    """Largest lockstep group of the batched solves (0 or 1: one whole-solve graph per problem);
    returns the previous setting."""
    return int(load().iim_set_lockstep(int(max_group)))


def iim_profile_begin():
    _check(load().iim_profile_begin(), "iim_profile_begin")


def iim_profile_end(capacity: int = 128):
    """Per-kernel records [{name, launches, ms, bytes, flops}] since iim_profile_begin."""
    buf = (iim_kernel_stat * capacity)()
    n = load().iim_profile_end(buf, capacity)
    return [{"name": buf[k].name.decode(), "launches": buf[k].launches, "ms": buf[k].ms, "bytes": buf[k].bytes,
             "flops": buf[k].flops} for k in range(min(n, capacity))]


def iim_transport_rhs(g: Geometry, omega, ux, uy, u_b, Uinf, nu, rhs_out, omega_b_in=None, omega_b_out=None,
                      dgamma_out=None, stream=None):
    NXY = (g.grid.nx - 1) * (g.grid.ny - 1)
    f64 = torch.float64
    U = (_d * 2)(float(Uinf[0]), float(Uinf[1]))
    st = load().iim_transport_rhs(g.handle, _ptr(omega, f64, NXY, "omega"), _ptr(ux, f64, NXY, "ux"),
                                  _ptr(uy, f64, NXY, "uy"), _ptr(u_b, f64, 2 * g.n_control, "u_b"), U, float(nu),
                                  _ptr(omega_b_in, f64, g.n_control, "omega_b_in"),
                                  _ptr(omega_b_out, f64, g.n_control, "omega_b_out"), _ptr(rhs_out, f64, NXY, "rhs_out"),
                                  _ptr(dgamma_out, f64, g.n_bodies, "dgamma_out"), _stream(stream))
    _check(st, "iim_transport_rhs")


def iim_geometry_set_wall_condition(g: Geometry, kind: int, stream=None):
    """0 Dirichlet ghost stencils (default), 1 Neumann (the psi_b argument of the solves is then
    the derivative along each control point's grid line into the fluid)."""
    _check(load().iim_geometry_set_wall_condition(g.handle, int(kind), _stream(stream)),
           "iim_geometry_set_wall_condition")


def iim_total_pressure_problem(g: Geometry, omega, ux, uy, u_b, Uinf, nu, f_out, data_out, omega_b_in=None,
                               omega_b_out=None, stream=None):
    """Right-hand side f and Neumann wall datum of the total-pressure problem (Sec. 5.4)."""
    NXY = (g.grid.nx - 1) * (g.grid.ny - 1)
    f64 = torch.float64
    U = (_d * 2)(float(Uinf[0]), float(Uinf[1]))
    st = load().iim_total_pressure_problem(g.handle, _ptr(omega, f64, NXY, "omega"), _ptr(ux, f64, NXY, "ux"),
                                           _ptr(uy, f64, NXY, "uy"), _ptr(u_b, f64, 2 * g.n_control, "u_b"), U,
                                           float(nu), _ptr(omega_b_in, f64, g.n_control, "omega_b_in"),
                                           _ptr(omega_b_out, f64, g.n_control, "omega_b_out"),
                                           _ptr(f_out, f64, NXY, "f_out"), _ptr(data_out, f64, g.n_control, "data_out"),
                                           _stream(stream))
    _check(st, "iim_total_pressure_problem")


def iim_wall_values(g: Geometry, field, out, stream=None):
    """A field (interior array) extrapolated to every control point."""
    NXY = (g.grid.nx - 1) * (g.grid.ny - 1)
    st = load().iim_wall_values(g.handle, _ptr(field, torch.float64, NXY, "field"),
                                _ptr(out, torch.float64, g.n_control, "out"), _stream(stream))
    _check(st, "iim_wall_values")


def iim_total_pressure(g: Geometry, omega, ux, uy, Uinf, nu, H_out, H_box=None, H_wall_out=None,
                       opts: iim_opts | None = None, stream=None, check=True):
    """The global surface-pressure method (Sec. 5.4) on a geometry in Neumann mode; returns the
    solve's iim_stats as a dict."""
    NXY = (g.grid.nx - 1) * (g.grid.ny - 1)
    f64 = torch.float64
    U = (_d * 2)(float(Uinf[0]), float(Uinf[1]))
    stats = iim_stats()
    o = opts if opts is not None else default_opts()
    st = load().iim_total_pressure(g.handle, _ptr(omega, f64, NXY, "omega"), _ptr(ux, f64, NXY, "ux"),
                                   _ptr(uy, f64, NXY, "uy"), U, float(nu),
                                   _ptr(H_box, f64, 2 * (g.grid.nx + g.grid.ny), "H_box"),
                                   _ptr(H_out, f64, NXY, "H_out"), _ptr(H_wall_out, f64, g.n_control, "H_wall_out"),
                                   ctypes.byref(o), ctypes.byref(stats), _stream(stream))
    d = stats.as_dict()
    d["status"] = st
    if check:
        _check(st, "iim_total_pressure")
    return d


def iim_rk3_step(g: Geometry, omega, gamma, psibar, u_b, psi_b, psi_box, Uinf, nu, c_stab, dt=0.0,
                 opts: iim_opts | None = None, stream=None, check=True):
    """One RK3 step in place on omega, gamma, psibar; returns (dt used, [stats per stage], status)."""
    NXY = (g.grid.nx - 1) * (g.grid.ny - 1)
    f64 = torch.float64
    U = (_d * 2)(float(Uinf[0]), float(Uinf[1]))
    dtc = _d(float(dt))
    stats = (iim_stats * 3)()
    o = opts if opts is not None else default_opts()
    st = load().iim_rk3_step(g.handle, _ptr(omega, f64, NXY, "omega"), _ptr(gamma, f64, g.n_bodies, "gamma"),
                             _ptr(psibar, f64, g.n_bodies, "psibar"), _ptr(u_b, f64, 2 * g.n_control, "u_b"),
                             _ptr(psi_b, f64, g.n_control, "psi_b"),
                             _ptr(psi_box, f64, 2 * (g.grid.nx + g.grid.ny), "psi_box"), U, float(nu), float(c_stab),
                             ctypes.byref(dtc), ctypes.byref(o), stats, _stream(stream))
    if check:
        _check(st, "iim_rk3_step")
    return dtc.value, [stats[k].as_dict() for k in range(3)], st


def iim_rk3_step_moving_wall(g: Geometry, omega, gamma, psibar, u_b, u_b_rate, psi_b, psi_box, Uinf, nu, c_stab,
                             dt=0.0, opts: iim_opts | None = None, stream=None, check=True):
    """iim_rk3_step with the wall velocity u_b + c dt u_b_rate at each stage time t + c dt."""
    NXY = (g.grid.nx - 1) * (g.grid.ny - 1)
    f64 = torch.float64
    U = (_d * 2)(float(Uinf[0]), float(Uinf[1]))
    dtc = _d(float(dt))
    stats = (iim_stats * 3)()
    o = opts if opts is not None else default_opts()
    st = load().iim_rk3_step_moving_wall(
        g.handle, _ptr(omega, f64, NXY, "omega"), _ptr(gamma, f64, g.n_bodies, "gamma"),
        _ptr(psibar, f64, g.n_bodies, "psibar"), _ptr(u_b, f64, 2 * g.n_control, "u_b"),
        _ptr(u_b_rate, f64, 2 * g.n_control, "u_b_rate"), _ptr(psi_b, f64, g.n_control, "psi_b"),
        _ptr(psi_box, f64, 2 * (g.grid.nx + g.grid.ny), "psi_box"), U, float(nu), float(c_stab), ctypes.byref(dtc),
        ctypes.byref(o), stats, _stream(stream))
    if check:
        _check(st, "iim_rk3_step_moving_wall")
    return dtc.value, [stats[k].as_dict() for k in range(3)], st
