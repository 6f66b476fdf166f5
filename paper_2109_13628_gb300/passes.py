"""Times the three passes of the rectangular solve (forward row transforms, column pass, inverse
row transforms) on the single-cylinder workload's grid through iim_time_box_passes, and prints
one JSON line: microseconds and algorithmic bytes per launch, and the column pass used.

    python -m paper_2109_13628_gb300.passes --n 1024 --col 1 --batch 40

--col: 1 tridiagonal scans, 0 column DSTs; --batch: fields per launch of each pass (forward rows,
column pass, inverse rows); --prec: mixed (FP32 transforms) or fp64.  Used to profile one pass in
isolation."""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import binding as iim
from . import inputs


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--col", type=int, default=1)
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--tiles", type=int, default=8)
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
    a = ap.parse_args(argv)
    P = inputs.c1_cylinder(a.n)
    g = P.grid
    dev = torch.device("cuda", 0)
    geo = iim.iim_setup_geometry(iim.make_grid(g.x0, g.x1, g.y0, g.y1, g.nx, g.ny),
                                 torch.as_tensor(np.ascontiguousarray(P.phi), dtype=torch.float64, device=dev),
                                 P.regions, P.modes)
    iim.iim_geometry_set_column_solver(geo, a.col)
    iim.iim_geometry_set_tiles(geo, a.tiles)
    r = iim.iim_time_box_passes(geo, iim.IIM_MIXED if a.prec == "mixed" else iim.IIM_FP64, a.batch, a.reps)
    print(json.dumps({"n": a.n, "column_pass": ["column DSTs", "tridiagonal scans"][a.col], "batch": a.batch,
                      "prec": a.prec, "passes": ["rows_fwd", "cols", "rows_inv"], **r}))
    geo.close()


if __name__ == "__main__":
    main()
