"""Pins of the oracle's network (definition of a dilated 3x3 convolution, its gradients)."""
import numpy as np

from oracle import net


def test_delta_response_is_the_flipped_kernel():
    """A unit impulse at (i0, j0) gives y[i0 - d(ky-1), j0 - d(kx-1)] = W[ky, kx]."""
    rng = np.random.default_rng(0)
    w = rng.normal(size=(1, 1, 3, 3))
    for d in (1, 3):
        x = np.zeros((1, 1, 13, 13))
        x[0, 0, 6, 6] = 1.0
        y = net.conv2d(x, w, np.zeros(1), d)
        for ky in range(3):
            for kx in range(3):
                assert y[0, 0, 6 - d * (ky - 1), 6 - d * (kx - 1)] == w[0, 0, ky, kx]
        assert np.count_nonzero(y) == 9


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    dils = [1, 2, 1]
    shapes = [(4, 2), (4, 4), (1, 4)]
    params = [(0.3 * rng.normal(size=(o, c, 3, 3)), 0.1 * rng.normal(size=o)) for o, c in shapes]
    x = rng.normal(size=(2, 2, 9, 8))
    target = rng.normal(size=(2, 1, 9, 8))
    mask = (rng.random(size=(2, 1, 9, 8)) > 0.2).astype(float)
    loss, grads = net.loss_and_grad(params, dils, x, target, mask)
    eps = 1e-6
    for li in range(3):
        for which in (0, 1):
            arr = params[li][which]
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(5, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp, _ = net.loss_and_grad(params, dils, x, target, mask)
                flat[idx] = old - eps
                lm, _ = net.loss_and_grad(params, dils, x, target, mask)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                an = grads[li][which].reshape(-1)[idx]
                assert abs(fd - an) < 1e-6 * max(1.0, abs(fd)), (li, which, fd, an)


def test_adam_first_step_moves_by_lr_in_sign_direction():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = net.adam_update(p, g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(p - p1, 0.01 * np.sign(g), rtol=1e-4)
