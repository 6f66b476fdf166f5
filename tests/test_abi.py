"""The C ABI library loads without a GPU and exports every function include/iim.h declares."""
import os
import re

from paper_2109_13628_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(iim_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("iim_setup_geometry", "iim_poisson_solve", "iim_destroy_geometry", "iim_box_poisson"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = binding.load()
    for n in sorted(declared_functions()):
        assert hasattr(lib, n), n
    assert {s[0] for s in binding.SIGNATURES} == declared_functions()


def test_status_strings_without_gpu():
    lib = binding.load()
    assert lib.iim_status_string(0) == b"IIM_OK"
    assert lib.iim_status_string(-2) == b"IIM_ERR_UNDERRESOLVED"
    assert lib.iim_status_string(123) == b"IIM_UNKNOWN_STATUS"


def test_invalid_arguments_rejected_before_any_cuda_call():
    import ctypes
    lib = binding.load()
    out = ctypes.c_void_p()
    g = binding.make_grid(0, 1, 0, 1, 100, 64)        # nx not a power of two
    assert lib.iim_setup_geometry(ctypes.byref(g), ctypes.c_void_p(8), 0, None, None, None, ctypes.byref(out)) == -1
    assert lib.iim_poisson_solve(None, None, None, None, None, None, None, None, None, None, None, None, None) == -1
    assert lib.iim_geometry_set_wall_condition(None, 1, None) == -1
    U = (ctypes.c_double * 2)(0.0, 0.0)
    assert lib.iim_total_pressure_problem(None, None, None, None, None, U, 0.0, None, None, None, None, None) == -1
    assert lib.iim_wall_values(None, None, None, None) == -1
    assert lib.iim_total_pressure(None, None, None, None, U, 0.0, None, None, None, None, None, None) == -1
    on, t = ctypes.c_int(), ctypes.c_int()
    assert lib.iim_net_set_tensor_cores(None, 1) == -1
    assert lib.iim_net_tensor_core_status(None, ctypes.byref(on), ctypes.byref(t)) == -1
