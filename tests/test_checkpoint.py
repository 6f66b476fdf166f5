"""Checkpoint format (host only): arrays come back byte for byte, the header carries t, the
step, the grid and the metadata, and truncated or foreign files are refused."""
import json

import numpy as np
import pytest
import torch

from paper_2109_13628_gb300 import checkpoint, inputs


def test_round_trip_is_exact(tmp_path):
    rng = np.random.default_rng(3)
    arrays = {"omega": torch.from_numpy(rng.normal(size=(63, 127))),
              "gamma": torch.tensor([1.25, -3e-17, np.pi]),
              "psibar": torch.tensor([0.0, -0.0, 7.5]),
              "flags": torch.tensor([1, 2, 3], dtype=torch.int32),
              "f32": torch.from_numpy(rng.normal(size=5).astype(np.float32))}
    g = inputs.square_grid(128)
    p = str(tmp_path / "state")
    checkpoint.save(p, arrays, t=1.5, step=42, grid=g, meta={"nu": 0.005})
    back, hdr = checkpoint.load(p)
    assert hdr["t"] == 1.5 and hdr["step"] == 42 and hdr["meta"] == {"nu": 0.005}
    assert hdr["grid"]["nx"] == 128 and hdr["grid"]["x0"] == -2.0
    for k, v in arrays.items():
        assert back[k].dtype == v.dtype and back[k].shape == v.shape
        assert back[k].numpy().tobytes() == v.numpy().tobytes(), k   # bitwise, signed zeros included
    raw = open(p + ".bin", "rb").read()
    assert raw[:8] == np.array([arrays["omega"][0, 0].item()], dtype="<f8").tobytes()   # little-endian


def test_refuses_truncated_and_foreign(tmp_path):
    p = str(tmp_path / "s")
    checkpoint.save(p, {"a": torch.arange(10, dtype=torch.float64)}, t=0.0, step=0)
    with open(p + ".bin", "r+b") as fh:
        fh.truncate(40)
    with pytest.raises(ValueError):
        checkpoint.load(p)
    checkpoint.save(p, {"a": torch.arange(10, dtype=torch.float64)}, t=0.0, step=0)
    hdr = json.load(open(p + ".json"))
    hdr["format"] = "something-else"
    json.dump(hdr, open(p + ".json", "w"))
    with pytest.raises(ValueError):
        checkpoint.load(p)
