"""FP64 CPU oracle of the neural-operator surrogate of the ph-ph collision integral.

TEST INFRASTRUCTURE ONLY (used by tests/ and bench.py's baseline legs; never by the
product path).  The paper has no learned component; this is the learned stand-in for
I^{ph-ph} (Eq. ph-ph) on the phonon sub-lattice used inside the MRI slow stage.

Network (one sample = the phonon populations of the nq_s x nq_s sub-lattice, one channel
per branch; periodic boundary conditions):
    x   = (N - mu) / sd                      per channel, mu/sd fixed from training data
    h1  = tanh(conv3x3(x;  W1, b1))          C_in -> width, circular padding
    h2  = tanh(conv3x3(h1; W2, b2))          width -> width
    h3  = tanh(conv3x3(h2; W3, b3))
    h4  = tanh(conv3x3(h3; W4, b4))
    h5  = tanh(h4 @ M1 + c1)                 pointwise width -> width
    out = h5 @ M2 + c2                       pointwise width -> C_out
    I   = out * so                           per-channel output scale
Loss = mean((out - I_target / so)^2) over points, channels and samples.

Convolution weight layout: W[tap, c_in, c_out] with tap = (dy + 1) * 3 + (dx + 1),
dy, dx in {-1, 0, 1}; out[y, x, co] = b[co] + sum_{tap, ci} in[(y+dy) % ny, (x+dx) % nx, ci] W[tap, ci, co].
Arrays are [batch, ny, nx, channels].  Parity unpinned for the design choices (they are the
build's own, not the paper's); the arithmetic is pinned by finite differences in
tests/test_oracle_surrogate.py.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def init_params(c_in: int, c_out: int, width: int, seed: int) -> dict:
    rng = np.random.default_rng(seed)
    p = {}
    chans = [c_in, width, width, width, width]
    for i in range(4):
        fan = 9 * chans[i]
        p[f"W{i + 1}"] = rng.standard_normal((9, chans[i], chans[i + 1])) / np.sqrt(fan)
        p[f"b{i + 1}"] = np.zeros(chans[i + 1])
    p["M1"] = rng.standard_normal((width, width)) / np.sqrt(width)
    p["c1"] = np.zeros(width)
    p["M2"] = rng.standard_normal((width, c_out)) / np.sqrt(width) * 0.1
    p["c2"] = np.zeros(c_out)
    return p


def conv(x, W, b):
    """x [B, ny, nx, ci], W [9, ci, co] -> [B, ny, nx, co] with periodic padding."""
    out = np.zeros(x.shape[:3] + (W.shape[2],))
    for t, (dy, dx) in enumerate(TAPS):
        xs = np.roll(x, shift=(-dy, -dx), axis=(1, 2))  # xs[y, x] = x[y + dy, x + dx]
        out += xs @ W[t]
    return out + b


def conv_backward(x, W, g):
    """Gradients of sum(g * conv(x, W, b)) w.r.t. x, W, b."""
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    B, ny, nx, ci = x.shape
    for t, (dy, dx) in enumerate(TAPS):
        xs = np.roll(x, shift=(-dy, -dx), axis=(1, 2))
        gW[t] = xs.reshape(-1, ci).T @ g.reshape(-1, g.shape[3])
        gx += np.roll(g @ W[t].T, shift=(dy, dx), axis=(1, 2))
    gb = g.reshape(-1, g.shape[3]).sum(axis=0)
    return gx, gW, gb


def forward(p: dict, x: np.ndarray):
    """Normalised input x -> normalised output, with the activations kept for backward."""
    cache = {"a0": x}
    a = x
    for i in range(1, 5):
        a = np.tanh(conv(a, p[f"W{i}"], p[f"b{i}"]))
        cache[f"a{i}"] = a
    a5 = np.tanh(a @ p["M1"] + p["c1"])
    cache["a5"] = a5
    out = a5 @ p["M2"] + p["c2"]
    return out, cache


def loss_and_grads(p: dict, x: np.ndarray, t: np.ndarray):
    """Mean-square loss against normalised targets t and its gradients."""
    out, c = forward(p, x)
    n = out.size
    d = out - t
    loss = float(np.sum(d * d) / n)
    g_out = 2.0 * d / n
    g = {}
    a5 = c["a5"]
    g["M2"] = a5.reshape(-1, a5.shape[-1]).T @ g_out.reshape(-1, g_out.shape[-1])
    g["c2"] = g_out.reshape(-1, g_out.shape[-1]).sum(axis=0)
    ga5 = g_out @ p["M2"].T
    gz5 = ga5 * (1.0 - a5 * a5)
    a4 = c["a4"]
    g["M1"] = a4.reshape(-1, a4.shape[-1]).T @ gz5.reshape(-1, gz5.shape[-1])
    g["c1"] = gz5.reshape(-1, gz5.shape[-1]).sum(axis=0)
    ga = gz5 @ p["M1"].T
    for i in range(4, 0, -1):
        ai = c[f"a{i}"]
        gz = ga * (1.0 - ai * ai)
        gx, gW, gb = conv_backward(c[f"a{i - 1}"], p[f"W{i}"], gz)
        g[f"W{i}"], g[f"b{i}"] = gW, gb
        ga = gx
    return loss, g


def predict(p: dict, N: np.ndarray, mu: np.ndarray, sd: np.ndarray, so: np.ndarray) -> np.ndarray:
    out, _ = forward(p, (N - mu) / sd)
    return out * so
