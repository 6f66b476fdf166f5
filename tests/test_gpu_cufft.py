"""The library's hand-written DST-I box solve against a cuFFT-based one (torch.fft; the timed
library cross-check of the benchmark).  cuFFT never enters the library: it is only the second
opinion here.  Sizes span the register-path FFT (1024-point lines), the Stockham path (2048) and
a ragged rectangle.  FP32 tolerances: the rounding error of an FP32 transform pair grows with
the line length, 2e-5 of the field's maximum up to 1024-point lines (the bound of the other box
tests), 5e-5 for 2048-point lines."""
import numpy as np
import pytest
import torch

import bench
import paper_2109_13628_gb300 as iim
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nx,ny", [(1024, 1024), (2048, 2048), (256, 64)])
def test_box_solve_agrees_with_cufft(nx, ny):
    h = 1.0 / 128
    g = iim.make_grid(0, nx * h, 0, ny * h, nx, ny)
    rng = np.random.default_rng(nx + 3 * ny)
    f = torch.as_tensor(rng.normal(size=(ny - 1, nx - 1)), dtype=torch.float64, device=gu.dev())
    ref = bench.cufft_box_poisson(f, h)
    scale = ref.abs().max().item()
    work = torch.empty(2 * f.numel(), dtype=torch.float64, device=gu.dev())
    tol32 = 2e-5 if max(nx, ny) <= 1024 else 5e-5
    for prec, tol in ((iim.IIM_FP64, 1e-12), (iim.IIM_MIXED, tol32)):
        u = torch.empty(f.numel(), dtype=torch.float64, device=gu.dev())
        iim.iim_box_poisson(g, f.reshape(-1), None, u, prec, work)
        err = (u.reshape(f.shape) - ref).abs().max().item() / scale
        assert err < tol, (prec, err)
    # the FP32 cuFFT solve sits within the same band of the FP64 one
    r32 = bench.cufft_box_poisson(f.float(), h).double()
    assert (r32 - ref).abs().max().item() / scale < tol32
