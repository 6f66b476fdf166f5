"""The learned guess: GPU forward/backward against the numpy oracle network (same BF16-rounded
weights, FP32 layer inputs and FP32 accumulation on the GPU: the CUDA-core kernels; the
tensor-core path has its own tests), training, and what the trained net gains."""
import numpy as np
import pytest
import torch

import paper_2109_13628_gb300 as iim
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
        w = flat[o:o + co * ci * 9].reshape(co, ci, 3, 3).astype(np.float64)
        o += co * ci * 9
        b = flat[o:o + co].astype(np.float64)
        o += co
        params.append((w, b))
    return params


@pytest.mark.parametrize("hidden,dils", [(8, (1, 2, 1)), (32, (1, 2, 4, 8, 16, 1))])
def test_forward_and_gradients_match_oracle(hidden, dils):
    dev = torch.device("cuda", 0)
    net = learned.Net(in_channels=3, hidden=hidden, dilations=dils, seed=3, tensor_cores=False)
    rng = np.random.default_rng(0)
    p = (0.3 * rng.normal(size=net.n)).astype(np.float32)
    net.set(p)
    params = unpack(p, 3, hidden, len(dils))
    params_q = [(bf16_round(w).astype(np.float64), b) for w, b in params]   # the GPU computes with BF16 weights
    x = rng.normal(size=(2, 3, 37, 45)).astype(np.float32)
    dy = rng.normal(size=(2, 1, 37, 45)).astype(np.float32)
    xt = torch.as_tensor(x, device=dev)
    y = torch.empty((2, 1, 37, 45), dtype=torch.float32, device=dev)
    net.forward(xt, y)
    acts = onet.forward(params_q, list(dils), x.astype(np.float64))
    ref = acts[-1]
    assert np.abs(y.cpu().numpy() - ref).max() < 2e-4 * np.abs(ref).max()
    g = net.backward(xt, torch.as_tensor(dy, device=dev))
    # oracle gradient of sum(dy * pred): loss_and_grad with target = pred - dy/2, mask = 1 gives 2 diff / N ...
    # so differentiate directly instead
    gout = dy.astype(np.float64)
    grads, gcur = [None] * len(dils), gout
    for li in range(len(dils) - 1, -1, -1):
        if li < len(dils) - 1:
            gcur = gcur * (acts[li + 1] > 0)
        gx, gw, gb = onet.conv2d_backward(acts[li], params_q[li][0], dils[li], gcur)
        grads[li] = (gw, gb)
        gcur = gx
    flat_ref = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])
    scale = np.abs(flat_ref).max()
    assert np.abs(g - flat_ref).max() < 2e-3 * scale, np.abs(g - flat_ref).max() / scale
    net.close()


def test_training_reduces_loss():
    dev = torch.device("cuda", 0)
    net = learned.Net(in_channels=3, hidden=8, dilations=(1, 2, 1), seed=1)
    rng = np.random.default_rng(2)
    x = torch.as_tensor(rng.normal(size=(4, 3, 32, 32)).astype(np.float32), device=dev)
    # a target the net can represent: a fixed smoothing of channel 0
    t = torch.nn.functional.avg_pool2d(x[:, :1], 3, stride=1, padding=1).contiguous()
    m = torch.ones_like(t)
    losses = [net.train_step(x, t, m, 3e-3) for _ in range(150)]
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])
    net.close()


def test_krylov_seed_from_exact_solution():
    """guess = 2 with the converged streamfunction as the guess: the seed leaves a small part of
    ||b|| and the first correction (the one the seed starts) needs fewer Krylov iterations than
    from zero.  Later corrections, e.g. one that only polishes the circulation rows, are not
    what the seed acts on."""
    dev = torch.device("cuda", 0)
    P = learned.training_problem(64, 90000)
    for prec in (iim.IIM_FP64, iim.IIM_MIXED):
        psi, st0 = learned.solve_problem(P, dev, prec=prec)
        psi1, st1 = learned.solve_problem(P, dev, prec=prec, guess=psi.clone())
        assert st0["seed_rel_res"] == 1.0
        assert st1["seed_rel_res"] < 0.1 and not st1["fallback"]
        assert st1["iters_first"] < st0["iters_first"]
        assert st1["rel_res"] <= 1e-10
        assert (psi1 - psi).abs().max().item() <= 1e-8 * psi.abs().max().item()


def test_learned_guess_on_unseen_problems():
    """Trained on the method's own solves (64^2, grid symmetries as augmentation), evaluated on
    unseen problems.  What the trained net gives, asserted as measured: its seed lowers the
    first correction's starting residual (0.73 of ||b|| on average in the last GPU run, against
    1 from zero; the seed is scaled to minimise that residual, so it never starts above ||b||),
    and the solve still meets the FP64 target.  It does not save Krylov iterations (17.3 per
    first correction against 17.7 from zero and 16.8 from the body-free box solve in that run):
    the iterations are printed, not asserted."""
    dev = torch.device("cuda", 0)
    data = learned.make_dataset(96, 64, 1000, dev)
    net = learned.Net(seed=5)
    losses = learned.train(net, data, epochs=30, batch=8, lr=2e-3)
    assert np.mean(losses[-10:]) < 0.1 * losses[0]
    it0, itb, it1, seeds = [], [], [], []
    k, seed = 0, 90000
    while k < 6:
        P = learned.training_problem(64, seed)
        seed += 1
        try:
            _, st0 = learned.solve_problem(P, dev)
        except iim.IIMError:
            continue
        S = learned.Sample(P, dev)
        _, stb = learned.solve_problem(P, dev, guess=S.ubox)
        _, st1 = learned.solve_problem(P, dev, guess=S.guess(net, dev))
        assert st1["rel_res"] <= 1e-10
        assert st1["seed_rel_res"] <= 1.0
        it0.append(st0["iters_first"])
        itb.append(stb["iters_first"])
        it1.append(st1["iters_first"])
        seeds.append(st1["seed_rel_res"])
        k += 1
    print(f"first-correction iterations: zero guess {np.mean(it0):.1f}, body-free box solve {np.mean(itb):.1f}, "
          f"learned guess {np.mean(it1):.1f}; learned seed residual / ||b|| {np.mean(seeds):.3f}")
    assert np.mean(seeds) < 0.9
    net.close()
