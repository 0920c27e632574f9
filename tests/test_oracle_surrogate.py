"""Pins for the FP64 oracle of the neural-operator surrogate: the periodic convolution
against an explicit-index loop, and every gradient against central finite differences."""
import numpy as np
import pytest

from oracle import surrogate_oracle as so


def test_periodic_conv_matches_explicit_indices():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 4, 5, 3))
    W = rng.standard_normal((9, 3, 2))
    b = rng.standard_normal(2)
    got = so.conv(x, W, b)
    B, ny, nx, _ = x.shape
    ref = np.zeros((B, ny, nx, 2))
    for n in range(B):
        for y in range(ny):
            for xx in range(nx):
                acc = b.copy()
                for t, (dy, dx) in enumerate(so.TAPS):
                    acc += x[n, (y + dy) % ny, (xx + dx) % nx] @ W[t]
                ref[n, y, xx] = acc
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("seed", [1, 2])
def test_gradients_match_central_differences(seed):
    rng = np.random.default_rng(seed)
    p = so.init_params(c_in=2, c_out=2, width=4, seed=seed)
    for k in p:  # non-zero biases so every term is exercised
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)
    x = rng.standard_normal((2, 4, 5, 2))
    t = rng.standard_normal((2, 4, 5, 2))
    loss, g = so.loss_and_grads(p, x, t)
    eps = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, min(flat.size, 6), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + eps
            lp, _ = so.loss_and_grads(p, x, t)
            flat[i] = old - eps
            lm, _ = so.loss_and_grads(p, x, t)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            an = g[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, i, fd, an)


def test_training_reduces_loss():
    """A few gradient steps on a fixed linear map of the inputs lower the loss (sanity of
    signs: a gradient with a wrong sign would raise it)."""
    rng = np.random.default_rng(3)
    p = so.init_params(c_in=2, c_out=2, width=8, seed=3)
    x = rng.standard_normal((4, 6, 6, 2))
    t = 0.5 * x[..., ::-1] + 0.1 * np.roll(x, 1, axis=1)
    l0, _ = so.loss_and_grads(p, x, t)
    for _ in range(60):
        _, g = so.loss_and_grads(p, x, t)
        for k in p:
            p[k] -= 0.2 * g[k]
    l1, _ = so.loss_and_grads(p, x, t)
    assert l1 < 0.3 * l0
