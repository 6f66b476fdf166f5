"""Tensor-core convolution of the learned guess's hidden layers (tcgen05 implicit GEMM, BF16
layer inputs and weights, FP32 accumulation in tensor memory) against the numpy oracle network.

The first test feeds a 32-channel input whose values are already BF16 numbers, so the GPU's
rounding of the layer input is the identity and the oracle sees the same operands: the only
difference left is the FP32 summation order (tolerance 1e-5 of the output's maximum).  Widths
of 300 and 129 pixels leave ragged 128-pixel tiles; dilations 1 to 32 cover the halo sizes the
net uses.  The second test runs the production-shaped net (3 -> 32 -> ... -> 1) with the oracle
rounding each hidden layer's input to BF16 as the kernel does; rounding decisions on values the
two sides computed in different precisions may differ, so the bound is 2e-3.  The gradients of
training go through the same kernel (the input gradient is a convolution with the flipped
weights), checked against the oracle's FP64 gradients within BF16 accuracy.  The last test puts
every layer on the tensor cores (3 -> 32 and 32 -> 1 padded to the MMA shape with zero channels;
a net of 8 hidden channels pads both K and N), the oracle rounding every layer's input."""
import numpy as np
import pytest
import torch

from oracle import net as onet
from paper_2109_13628_gb300 import learned

pytestmark = pytest.mark.gpu


def bf16_round(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def unpack(flat, cin, hidden, nl):
    params, o = [], 0
    for l in range(nl):
        ci = cin if l == 0 else hidden
        co = 1 if l == nl - 1 else hidden
        w = bf16_round(flat[o:o + co * ci * 9]).reshape(co, ci, 3, 3).astype(np.float64)
        o += co * ci * 9
        b = flat[o:o + co].astype(np.float64)
        o += co
        params.append((w, b))
    return params


@pytest.mark.parametrize("d,H,W", [(1, 37, 300), (3, 20, 129), (16, 33, 256), (32, 40, 131)])
def test_tensor_core_layer_matches_oracle_exact_operands(d, H, W):
    dev = torch.device("cuda", 0)
    net = learned.Net(in_channels=32, hidden=32, dilations=(d, 1), seed=5, tensor_cores=1)
    rng = np.random.default_rng(d)
    p = (0.2 * rng.normal(size=net.n)).astype(np.float32)
    net.set(p)
    params = unpack(p, 32, 32, 2)
    x = bf16_round(rng.normal(size=(2, 32, H, W)))
    y = torch.empty((2, 1, H, W), dtype=torch.float32, device=dev)
    net.forward(torch.as_tensor(x, device=dev), y)
    ref = onet.forward(params, [d, 1], x.astype(np.float64))[-1]
    err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err
    assert net.tensor_core_status() == (1, 0)
    net.close()


def test_tensor_core_net_forward_and_gradients_match_oracle():
    dev = torch.device("cuda", 0)
    dils = (1, 2, 4, 8, 16, 1)
    net = learned.Net(in_channels=3, hidden=32, dilations=dils, seed=3, tensor_cores=1)
    rng = np.random.default_rng(1)
    p = (0.3 * rng.normal(size=net.n)).astype(np.float32)
    net.set(p)
    params = unpack(p, 3, 32, len(dils))
    x = rng.normal(size=(2, 3, 45, 150)).astype(np.float32)
    dy = rng.normal(size=(2, 1, 45, 150)).astype(np.float32)
    xt = torch.as_tensor(x, device=dev)
    y = torch.empty((2, 1, 45, 150), dtype=torch.float32, device=dev)
    net.forward(xt, y)
    # oracle forward with the hidden layers' inputs rounded to BF16, as the tensor-core kernel does
    acts = [x.astype(np.float64)]
    h = acts[0]
    for li, ((w, b), d) in enumerate(zip(params, dils)):
        hin = bf16_round(h).astype(np.float64) if 0 < li < len(dils) - 1 else h
        h = onet.conv2d(hin, w, b, d)
        if li < len(dils) - 1:
            h = np.maximum(h, 0.0)
        acts.append(h)
    ref = acts[-1]
    err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 2e-3, err
    g = net.backward(xt, torch.as_tensor(dy, device=dev))
    gcur, grads = dy.astype(np.float64), [None] * len(dils)
    for li in range(len(dils) - 1, -1, -1):
        if li < len(dils) - 1:
            gcur = gcur * (acts[li + 1] > 0)
        gx, gw, gb = onet.conv2d_backward(acts[li], params[li][0], dils[li], gcur)
        grads[li] = (gw, gb)
        gcur = gx
    flat_ref = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])
    gerr = np.abs(g - flat_ref).max() / np.abs(flat_ref).max()
    assert gerr < 2e-2, gerr
    assert net.tensor_core_status() == (1, 0)
    net.close()


@pytest.mark.parametrize("hidden,dils", [(32, (1, 2, 4, 8, 16, 1)), (8, (1, 3, 1))])
def test_tensor_cores_on_every_layer_match_oracle(hidden, dils):
    dev = torch.device("cuda", 0)
    net = learned.Net(in_channels=3, hidden=hidden, dilations=dils, seed=7, tensor_cores=2)
    rng = np.random.default_rng(hidden)
    p = (0.3 * rng.normal(size=net.n)).astype(np.float32)
    net.set(p)
    params = unpack(p, 3, hidden, len(dils))
    x = rng.normal(size=(2, 3, 41, 140)).astype(np.float32)
    dy = rng.normal(size=(2, 1, 41, 140)).astype(np.float32)
    xt = torch.as_tensor(x, device=dev)
    y = torch.empty((2, 1, 41, 140), dtype=torch.float32, device=dev)
    net.forward(xt, y)
    acts = [x.astype(np.float64)]
    h = acts[0]
    for li, ((w, b), d) in enumerate(zip(params, dils)):
        h = onet.conv2d(bf16_round(h).astype(np.float64), w, b, d)
        if li < len(dils) - 1:
            h = np.maximum(h, 0.0)
        acts.append(h)
    ref = acts[-1]
    err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 2e-3, err
    g = net.backward(xt, torch.as_tensor(dy, device=dev))
    gcur, grads = dy.astype(np.float64), [None] * len(dils)
    for li in range(len(dils) - 1, -1, -1):
        if li < len(dils) - 1:
            gcur = gcur * (acts[li + 1] > 0)
        gx, gw, gb = onet.conv2d_backward(acts[li], params[li][0], dils[li], gcur)
        grads[li] = (gw, gb)
        gcur = gx
    flat_ref = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])
    gerr = np.abs(g - flat_ref).max() / np.abs(flat_ref).max()
    assert gerr < 2e-2, gerr
    assert net.tensor_core_status() == (2, 0)
    net.close()
