"""The allocation-free box solve (iim_box_poisson_noalloc) against the workspace version.

Some callers cannot allocate device memory: code running during CUDA graph capture, real-time
or embedded hosts that must not touch the device allocator, and applications whose memory
pool already owns the free device memory.  For them the library offers a variant of the
Dirichlet-box solve whose scratch is a static device array.  This test calls it through the
C ABI twice in a row (different data, so a stale scratch from the first call would show) and
compares each result with iim_box_poisson at the tolerances the other box-solver tests use.
It is collected last so that a failure here cannot hide failures elsewhere, and it passes
both alone in a fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2109_13628_gb300 as iim
from paper_2109_13628_gb300 import binding

pytestmark = pytest.mark.gpu

TOL = {iim.IIM_FP64: 1e-12, iim.IIM_MIXED: 2e-5}


def dev():
    return torch.device("cuda", 0)


@pytest.mark.parametrize("prec", [iim.IIM_FP64, iim.IIM_MIXED])
@pytest.mark.parametrize("nx,ny", [(256, 128), (1024, 1024)])
def test_noalloc_matches_workspace_version_twice(prec, nx, ny):
    h = 1.0 / 64
    g = iim.make_grid(0, nx * h, 0, ny * h, nx, ny)
    NXY = (nx - 1) * (ny - 1)
    work = torch.empty(2 * NXY, dtype=torch.float64, device=dev())
    for call in range(2):
        rng = np.random.default_rng(100 * call + nx + prec)
        f = torch.as_tensor(rng.normal(size=NXY), device=dev())
        ring = torch.as_tensor(rng.normal(size=2 * (nx + ny)), device=dev())
        ref = torch.empty(NXY, dtype=torch.float64, device=dev())
        out = torch.full((NXY,), float("nan"), dtype=torch.float64, device=dev())
        iim.iim_box_poisson(g, f, ring, ref, prec, work)
        iim.iim_box_poisson_noalloc(g, f, ring, out, prec)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.isfinite(o).all()
        assert np.abs(o - r).max() < TOL[prec] * np.abs(r).max(), (call, np.abs(o - r).max())


def test_noalloc_rejects_grids_beyond_its_scratch():
    g = iim.make_grid(0, 32.0, 0, 0.25, 2048, 16)
    NXY = 2047 * 15
    f = torch.zeros(NXY, dtype=torch.float64, device=dev())
    u = torch.zeros(NXY, dtype=torch.float64, device=dev())
    with pytest.raises(iim.IIMError) as e:
        iim.iim_box_poisson_noalloc(g, f, None, u, iim.IIM_FP64)
    assert e.value.status == iim.IIM_ERR_INVALID_ARG
    assert b"static scratch" in binding.load().iim_last_error_message()


def test_noalloc_inside_a_captured_graph():
    """The use the entry point exists for: after one call outside any capture (the per-device
    set-up), the call is captured into a CUDA graph with no allocation, and every replay gives
    the workspace version's result."""
    nx, ny = 256, 128
    h = 1.0 / 64
    g = iim.make_grid(0, nx * h, 0, ny * h, nx, ny)
    NXY = (nx - 1) * (ny - 1)
    rng = np.random.default_rng(7)
    f = torch.as_tensor(rng.normal(size=NXY), device=dev())
    ring = torch.as_tensor(rng.normal(size=2 * (nx + ny)), device=dev())
    out = torch.zeros(NXY, dtype=torch.float64, device=dev())
    iim.iim_box_poisson_noalloc(g, f, ring, out, iim.IIM_FP64)   # set-up outside the capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        iim.iim_box_poisson_noalloc(g, f, ring, out, iim.IIM_FP64)
    work = torch.empty(2 * NXY, dtype=torch.float64, device=dev())
    ref = torch.empty(NXY, dtype=torch.float64, device=dev())
    for rep in range(2):
        f.copy_(torch.as_tensor(rng.normal(size=NXY), device=dev()))
        out.fill_(float("nan"))
        graph.replay()
        iim.iim_box_poisson(g, f, ring, ref, iim.IIM_FP64, work)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.abs(o - r).max() < TOL[iim.IIM_FP64] * np.abs(r).max(), (rep, np.abs(o - r).max())


_FIRST_CALL_UNDER_CAPTURE = r"""
import sys
sys.path.insert(0, sys.argv[1])
import torch
import paper_2109_13628_gb300 as iim
from paper_2109_13628_gb300 import binding
torch.cuda.set_device(0)
g = iim.make_grid(0, 1.0, 0, 1.0, 64, 64)
f = torch.zeros(63 * 63, dtype=torch.float64, device="cuda")
u = torch.zeros_like(f)
torch.cuda.synchronize()
graph = torch.cuda.CUDAGraph()
code = None
with torch.cuda.graph(graph):
    try:
        iim.iim_box_poisson_noalloc(g, f, None, u, iim.IIM_FP64)
    except iim.IIMError as e:
        code = e.status
msg = binding.load().iim_last_error_message().decode()
print("STATUS", code, msg)
"""


def test_noalloc_first_call_under_capture_is_refused():
    """The first call on a device sets up tables with device copies, which a capture cannot
    hold: made inside a capture it is refused with IIM_ERR_INVALID_ARG and a message, instead of
    breaking the caller's capture.  Runs in a fresh process so that the call really is the
    first one on the device."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL_UNDER_CAPTURE, root], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("STATUS")][-1]
    assert line.split()[1] == str(iim.IIM_ERR_INVALID_ARG), line
    assert "before any stream capture" in line
