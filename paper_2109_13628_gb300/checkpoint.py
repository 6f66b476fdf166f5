"""Checkpoint and resume of a flow simulation's state.

The state the time integration carries from step to step (Sec. 5.5) is the vorticity omega,
the circulation Gamma_k of every circulation-mode body and the time t; psibar_k (the bodies'
streamfunction constants) is kept as well so that the next solve starts from the same
values.  A checkpoint is two files: `<path>.json`, a header with the format tag, t, the step
number, the grid, the caller's metadata and, per array, its name, dtype, shape and byte range;
and `<path>.bin`, the arrays' raw little-endian bytes back to back.  Loading returns the same
bytes, so a resumed run repeats the original run's next step bit for bit.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

FORMAT = "iim-flow-state-v1"
_DTYPES = {torch.float64: "<f8", torch.float32: "<f4", torch.int32: "<i4", torch.int64: "<i8"}
_TORCH = {v: k for k, v in _DTYPES.items()}


def save(path: str, arrays: dict, *, t: float, step: int, grid=None, meta: dict | None = None) -> None:
    """Writes `arrays` (name -> tensor on any device) and the header.  The header is written
    last, so a checkpoint whose header exists is complete."""
    entries, offset = [], 0
    tmp_bin = path + ".bin.tmp"
    with open(tmp_bin, "wb") as fh:
        for name, t_ in arrays.items():
            if t_.dtype not in _DTYPES:
                raise TypeError(f"{name}: unsupported dtype {t_.dtype}")
            a = t_.detach().to("cpu").contiguous().numpy().astype(_DTYPES[t_.dtype], copy=False)
            b = a.tobytes(order="C")
            fh.write(b)
            entries.append({"name": name, "dtype": _DTYPES[t_.dtype], "shape": list(a.shape), "offset": offset,
                            "nbytes": len(b)})
            offset += len(b)
    os.replace(tmp_bin, path + ".bin")
    header = {"format": FORMAT, "t": float(t), "step": int(step), "arrays": entries, "bytes": offset,
              "grid": None if grid is None else {k: getattr(grid, k) for k in ("x0", "x1", "y0", "y1", "nx", "ny")},
              "meta": meta or {}}
    tmp_json = path + ".json.tmp"
    with open(tmp_json, "w") as fh:
        json.dump(header, fh, indent=1)
    os.replace(tmp_json, path + ".json")


def load(path: str, device=None) -> tuple[dict, dict]:
    """Returns (arrays: name -> tensor on `device`, header).  Raises ValueError when the header
    is not this format or the data file does not match it."""
    with open(path + ".json") as fh:
        header = json.load(fh)
    if header.get("format") != FORMAT:
        raise ValueError(f"{path}: not a {FORMAT} checkpoint")
    size = os.path.getsize(path + ".bin")
    if size != header["bytes"]:
        raise ValueError(f"{path}: data file has {size} bytes, header says {header['bytes']}")
    raw = np.fromfile(path + ".bin", dtype=np.uint8)
    out = {}
    for e in header["arrays"]:
        dt = np.dtype(e["dtype"])
        n = int(np.prod(e["shape"])) if e["shape"] else 1
        if e["nbytes"] != n * dt.itemsize or e["offset"] + e["nbytes"] > size:
            raise ValueError(f"{path}: array {e['name']} does not fit its byte range")
        a = raw[e["offset"]:e["offset"] + e["nbytes"]].view(dt).reshape(e["shape"]).astype(dt.newbyteorder("="))
        t_ = torch.from_numpy(a.copy())
        out[e["name"]] = t_.to(device) if device is not None else t_
    return out, header
