"""Learned initial guess for the IIM Poisson iteration (binding of the iim_net_* entry points
plus the data pipeline).

The network sees three planes on the interior grid: the vorticity, the level set (signed
distance to the bodies) and the rectangular solve of the vorticity that ignores the bodies
(one Dirichlet-box DST solve); it predicts the scaled difference between the method's
solution and that rectangular solve, which is concentrated around the bodies.  Training pairs
come from the method itself (iim_poisson_solve).  The guess enters through iim_opts.guess = 2:
it seeds the Krylov unknowns of the first correction (the IIM corrections it implies), and
the solver keeps it only if it lowers the Krylov residual."""
from __future__ import annotations

import ctypes
import time

import numpy as np
import torch

from . import binding as B
from . import inputs

DILATIONS = (1, 2, 4, 8, 16, 1)
HIDDEN = 32
IN_CHANNELS = 3


class Net:
    def __init__(self, in_channels=IN_CHANNELS, hidden=HIDDEN, dilations=DILATIONS, seed=0, tensor_cores=2):
        lib = B.load()
        d = (ctypes.c_int * len(dilations))(*dilations)
        h = ctypes.c_void_p()
        B._check(lib.iim_net_create(in_channels, hidden, len(dilations), d, seed, ctypes.byref(h)), "iim_net_create")
        self.h = h
        self.n = int(lib.iim_net_num_params(h))
        self.dilations = tuple(dilations)
        self.set_tensor_cores(tensor_cores)

    def set_tensor_cores(self, on):
        """Convolutions on the tensor cores (BF16 layer inputs): 2 every layer, 1 (or True) the
        32 -> 32 layers only, 0 (or False) none (FP32 inputs on the CUDA cores)."""
        B._check(B.load().iim_net_set_tensor_cores(self.h, int(on)), "iim_net_set_tensor_cores")

    def tensor_core_status(self):
        """(setting, 1 if a tensor-core convolution ever timed out waiting for its MMAs)."""
        on, t = ctypes.c_int(), ctypes.c_int()
        B._check(B.load().iim_net_tensor_core_status(self.h, ctypes.byref(on), ctypes.byref(t)),
                 "iim_net_tensor_core_status")
        return on.value, t.value

    def close(self):
        if self.h:
            B.load().iim_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self):
        out = np.empty(self.n, dtype=np.float32)
        B._check(B.load().iim_net_get_params(self.h, out.ctypes.data_as(ctypes.c_void_p), self.n), "iim_net_get_params")
        return out

    def set(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        B._check(B.load().iim_net_set_params(self.h, p.ctypes.data_as(ctypes.c_void_p), self.n), "iim_net_set_params")

    def forward(self, x, y, stream=None):
        b, _, hh, ww = x.shape
        B._check(B.load().iim_net_forward(self.h, b, hh, ww, B._ptr(x, torch.float32), B._ptr(y, torch.float32),
                                          B._stream(stream)), "iim_net_forward")

    def backward(self, x, dy, stream=None):
        b, _, hh, ww = x.shape
        g = np.empty(self.n, dtype=np.float32)
        B._check(B.load().iim_net_backward(self.h, b, hh, ww, B._ptr(x, torch.float32), B._ptr(dy, torch.float32),
                                           g.ctypes.data_as(ctypes.c_void_p), B._stream(stream)), "iim_net_backward")
        return g

    def train_step(self, x, target, mask, lr, stream=None, want_loss=True):
        b, _, hh, ww = x.shape
        loss = ctypes.c_float()
        B._check(B.load().iim_net_train_step(self.h, b, hh, ww, B._ptr(x, torch.float32), B._ptr(target, torch.float32),
                                             B._ptr(mask, torch.float32), float(lr),
                                             ctypes.byref(loss) if want_loss else None, B._stream(stream)),
                 "iim_net_train_step")
        return loss.value


def scales(P):
    """Per-problem input / output scales: vorticity RMS, domain size."""
    L = P.grid.x1 - P.grid.x0
    s_w = 1.0 / max(float(np.sqrt(np.mean(P.omega ** 2))), 1e-30)
    return {"s_omega": s_w, "s_phi": 1.0 / L, "s_box": s_w / (L * L), "s_out": s_w / (L * L)}


class Sample:
    """Device tensors of one problem: the network input, the rectangular solve, the mask."""

    def __init__(self, P, dev, omega=None, phi=None, mask=True, box_prec=B.IIM_FP64):
        """omega / phi: device FP64 copies the caller already holds (else uploaded from P);
        mask: build the fluid mask (training only); box_prec: precision of the body-free box
        solve that feeds the net and the guess (IIM_MIXED = FP32 transforms)."""
        g = P.grid
        self.P = P
        self.grid = B.make_grid(g.x0, g.x1, g.y0, g.y1, g.nx, g.ny)
        self.sc = scales(P)
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
        self.omega = omega if omega is not None else T(P.omega.ravel())
        self.phi = phi if phi is not None else T(P.phi)
        n = P.omega.size
        self.ubox = torch.empty(n, dtype=torch.float64, device=dev)
        work = torch.empty(2 * n + 4 * g.nx, dtype=torch.float64, device=dev)
        B.iim_box_poisson(self.grid, self.omega, None, self.ubox, box_prec, work)
        self.x = torch.empty((1, IN_CHANNELS, g.ny - 1, g.nx - 1), dtype=torch.float32, device=dev)
        B._check(B.load().iim_net_prepare_input(g.nx, g.ny, B._ptr(self.omega), B._ptr(self.phi), B._ptr(self.ubox),
                                                self.sc["s_omega"], self.sc["s_phi"], self.sc["s_box"],
                                                B._ptr(self.x), B._stream(None)), "iim_net_prepare_input")
        self.mask = None
        if mask:
            self.mask = torch.as_tensor((P.phi[1:-1, 1:-1] >= 0).astype(np.float32),
                                        device=dev).reshape(1, 1, g.ny - 1, g.nx - 1)

    def guess(self, net, dev):
        g = self.P.grid
        y = torch.empty((1, 1, g.ny - 1, g.nx - 1), dtype=torch.float32, device=dev)
        net.forward(self.x, y)
        psi = torch.empty(self.P.omega.size, dtype=torch.float64, device=dev)
        B._check(B.load().iim_net_compose_guess(psi.numel(), B._ptr(self.ubox), B._ptr(y), self.sc["s_out"],
                                                B._ptr(psi), B._stream(None)), "iim_net_compose_guess")
        return psi


def training_problem(n, seed):
    """A training / evaluation problem: [-2,2]^2, 2-5 circles or ellipses, Gaussian vortices,
    bodies in circulation mode with Gamma = h^2 sum over R_k of omega."""
    rng = np.random.default_rng(seed)
    g = inputs.square_grid(n)
    X, Y = g.nodes()
    nb = int(rng.integers(2, 6))
    axes = rng.uniform(0.2, 0.5, size=(nb, 2))
    circle = rng.random(nb) < 0.5
    axes[circle, 1] = axes[circle, 0]
    angles = rng.uniform(0, np.pi, size=nb)
    while True:
        try:
            centers = inputs.separated_centers(rng, nb, -1.3, 1.3, list(axes[:nb].max(axis=1)), max(0.25, 8 * g.h))
            break
        except RuntimeError:
            nb -= 1                        # fewer bodies when the draw does not fit
    axes, angles = axes[:nb], angles[:nb]
    bodies = [inputs.phi_ellipse(X, Y, c[0], c[1], a[0], a[1], t) for c, a, t in zip(centers, axes, angles)]
    phi = inputs.union(*bodies)
    w = inputs.vortex_field(g, seed + 17, 50, 0.1)
    omega = np.where(phi >= 0, w, 0.0)[1:-1, 1:-1]
    return inputs.Problem(grid=g, phi=phi, regions=[inputs.region_around(g, b) for b in bodies], modes=[1] * nb,
                          omega=np.ascontiguousarray(omega), psi_box=np.zeros(4 * n),
                          psi_b_fn=lambda x, y, k: np.zeros_like(x), psibar=np.zeros(nb), gamma=None, exact=None)


def gamma_of(P):
    h = P.grid.h
    return np.array([h * h * P.omega[r[2] - 1:r[3], r[0] - 1:r[1]].sum() for r in P.regions])


def solve_problem(P, dev, guess=None, prec=B.IIM_MIXED, rtol=1e-10, precond=0):
    """The method's solve of P (setup included); returns (psi, stats)."""
    g = P.grid
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    geo = B.iim_setup_geometry(B.make_grid(g.x0, g.x1, g.y0, g.y1, g.nx, g.ny), T(P.phi), P.regions, P.modes)
    try:
        psi = torch.empty(P.omega.size, dtype=torch.float64, device=dev)
        pb = torch.zeros(len(P.regions), dtype=torch.float64, device=dev)
        st = B.iim_poisson_solve(geo, T(P.omega.ravel()), T(np.zeros(geo.n_control)), None, T(gamma_of(P)), pb, psi,
                                 psi_guess=guess, opts=B.default_opts(prec=prec, rtol=rtol, guess=0 if guess is None else 2,
                                                                      precond=precond))
    finally:
        geo.close()
    return psi, st


def make_dataset(count, n, seed0, dev):
    """(inputs, targets, masks) stacked on the device, from `count` method solves at n^2."""
    xs, ts, ms = [], [], []
    k = 0
    seed = seed0
    while k < count:
        P = training_problem(n, seed)
        seed += 1
        try:
            psi, st = solve_problem(P, dev)
        except B.IIMError:
            continue                       # under-resolved draw
        S = Sample(P, dev)
        t = ((psi - S.ubox) * S.sc["s_out"]).to(torch.float32).reshape(1, 1, n - 1, n - 1)
        xs.append(S.x)
        ts.append(t)
        ms.append(S.mask)
        k += 1
    return torch.cat(xs), torch.cat(ts), torch.cat(ms)


def dihedral(a, k):
    """The k-th of the 8 symmetries of the square grid (k & 4: transpose, k & 1 / k & 2: flip the
    columns / rows) applied to (..., H, W) arrays.  The Poisson problem on a square box with
    zero box data commutes with all of them, so (input, target, mask) triples stay valid."""
    if k & 4:
        a = a.transpose(-1, -2)
    if k & 1:
        a = a.flip(-1)
    if k & 2:
        a = a.flip(-2)
    return a.contiguous()


def train(net, data, epochs, batch, lr, time_budget_s=None, seed=0, augment=True):
    """Adam on the masked mean-square error; each batch under a random grid symmetry."""
    x, t, m = data
    n = x.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = rng.permutation(n)
        for b0 in range(0, n - batch + 1, batch):
            idx = torch.as_tensor(perm[b0:b0 + batch], device=x.device)
            k = int(rng.integers(8)) if augment and x.shape[-1] == x.shape[-2] else 0
            losses.append(net.train_step(dihedral(x[idx], k), dihedral(t[idx], k), dihedral(m[idx], k), lr))
        if time_budget_s is not None and time.perf_counter() - t0 > time_budget_s:
            break
    return losses


def time_forward(n, batch=1, reps=10, tensor_cores=2, backward=False, seed=0):
    """Device milliseconds of one forward pass (and, with backward, of one backward pass) of the
    production net on batch x 3 x n x n random inputs: CUDA events around reps launches after
    three warm-up passes."""
    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device=dev).manual_seed(seed)
    x = torch.randn(batch, IN_CHANNELS, n, n, device=dev, generator=g)
    y = torch.empty(batch, 1, n, n, device=dev)
    net = Net(seed=seed, tensor_cores=tensor_cores)
    out = {}
    try:
        for _ in range(3):
            net.forward(x, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            net.forward(x, y)
        e1.record()
        torch.cuda.synchronize()
        out["forward_ms"] = e0.elapsed_time(e1) / reps
        # per-kernel split of one more forward pass (CUDA events around every launch)
        B.iim_profile_begin()
        net.forward(x, y)
        out["kernels"] = {r["name"]: {"launches": r["launches"], "ms": r["ms"],
                                      "gbs": r["bytes"] / (r["ms"] * 1e6) if r["ms"] > 0 else None,
                                      "tflops": r["flops"] / (r["ms"] * 1e9) if r["ms"] > 0 else None}
                          for r in B.iim_profile_end()}
        if backward:
            dy = torch.randn_like(y)
            net.backward(x, dy)
            t0 = time.perf_counter()
            for _ in range(3):
                net.backward(x, dy)   # synchronous (copies the gradient to the host)
            out["backward_ms_wall"] = (time.perf_counter() - t0) / 3 * 1e3
        out["tensor_cores"], out["timed_out"] = net.tensor_core_status()
    finally:
        net.close()
    return out


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="time the learned guess's network (forward, optional backward)")
    ap.add_argument("--n", type=int, default=1023)
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--tc", type=int, choices=[0, 1, 2], default=2)
    ap.add_argument("--backward", action="store_true")
    a = ap.parse_args()
    r = time_forward(a.n, a.batch, a.reps, a.tc, a.backward)
    print(json.dumps({"n": a.n, "batch": a.batch, **r}))
