"""FP64 reference of the learned correction -- TEST INFRASTRUCTURE.

The correction is not part of the paper: a small MLP maps a host's feature
vector (oracle.Oracle.features: 64-bin register histogram / g and sharing-
noise statistics, 80 inputs) to delta, and the corrected estimate is
n = exp(ln(1 + n_plain) + delta) - 1.  The training target is
delta* = ln(1 + c) - ln(1 + n_plain) for the exact cardinality c, the loss the
mean of (delta - delta*)^2.

This module holds the plain FP64 network (forward, backward) that pins the
library's BF16/FP32 kernels, and the generator of (features, exact
cardinality) training sets from oracle runs on trace-shaped traffic.

Network: x[80] -> GELU(W1 x + b1)[64] -> GELU(W2 h1 + b2)[64] -> w3 . h2 + b3,
GELU in its tanh form, z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).  Parameters in a flat float vector laid
out as W1 (64 x 80, row-major), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

IN, HID = 80, 64
SIZES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
         ("w3", (HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


GELU_A = np.sqrt(2.0 / np.pi)
GELU_B = 0.044715


def gelu(z):
    """GELU in its tanh form (Hendrycks & Gimpel 2016):
    z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))."""
    return 0.5 * z * (1.0 + np.tanh(GELU_A * (z + GELU_B * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_A * (z + GELU_B * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_A * (1.0 + 3.0 * GELU_B * z * z)


def gelu_exact(z):
    """z Phi(z), the definition the tanh form approximates."""
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def forward(theta: np.ndarray, X: np.ndarray):
    p = unpack(np.asarray(theta, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    d = h2 @ p["w3"] + p["b3"][0]
    return d, (X, z1, h1, z2, h2)


def loss(theta, X, y):
    d, _ = forward(theta, X)
    return float(np.mean((d - y) ** 2))


def gradient(theta, X, y) -> np.ndarray:
    """d loss / d theta (mean squared error over the batch), flat like theta."""
    p = unpack(np.asarray(theta, dtype=np.float64))
    d, (X, z1, h1, z2, h2) = forward(theta, X)
    g = 2.0 * (d - np.asarray(y, dtype=np.float64)) / d.size
    gw3 = h2.T @ g
    gb3 = np.array([g.sum()])
    dz2 = np.outer(g, p["w3"]) * gelu_grad(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, gb3])


def correct(n_plain, delta):
    return np.maximum(np.expm1(np.log1p(n_plain) + delta), 0.0)


# ------------------------------------------- the compact correction network
# A smaller network on ten features that the planned estimate can compute
# from a host's exact sums and four register counts, so that it runs inside
# the estimate's own kernel: the counts of register values 0..3 over g (the
# first four bins of the histogram above) and inputs 64..69 of the feature
# row (log2 g / 16, ln(1 + n_plain) / 16, ln(1 + n_g) / 16, ln(1 + n_Z / Z),
# V_Z / Z, V / g).  Network: x[10] -> GELU(W1 x + b1)[16] -> GELU(W2 h1 +
# b2)[16] -> w3 . h2 + b3, the same tanh-form GELU; parameters in a flat
# vector W1 (16 x 10, row-major), b1, W2 (16 x 16), b2, w3, b3.
C_IN, C_HID = 10, 16
C_SIZES = [("W1", (C_HID, C_IN)), ("b1", (C_HID,)), ("W2", (C_HID, C_HID)), ("b2", (C_HID,)),
           ("w3", (C_HID,)), ("b3", (1,))]
C_N_PARAMS = sum(int(np.prod(s)) for _, s in C_SIZES)


def compact_features(X80: np.ndarray) -> np.ndarray:
    """The ten inputs of the compact network from 80-input feature rows."""
    X80 = np.asarray(X80, dtype=np.float64)
    return np.concatenate([X80[:, 0:4], X80[:, 64:70]], axis=1)


def compact_forward(theta: np.ndarray, Xc: np.ndarray) -> np.ndarray:
    """delta of the compact network for rows Xc [n, 10], FP64."""
    th = np.asarray(theta, dtype=np.float64)
    p, o = {}, 0
    for name, shape in C_SIZES:
        k = int(np.prod(shape))
        p[name] = th[o:o + k].reshape(shape)
        o += k
    Xc = np.asarray(Xc, dtype=np.float64)
    h1 = gelu(Xc @ p["W1"].T + p["b1"])
    h2 = gelu(h1 @ p["W2"].T + p["b2"])
    return h2 @ p["w3"] + p["b3"][0]


# ------------------------------------------------------------- training sets

def trace_shaped_run(seed: int, scale: int = 16, slices: int | None = None):
    """One oracle run on trace-shaped traffic (Zipf 1.05, 10% in-slice repeats,
    k = 30, g = 256) at 1/scale of the pairs, hosts, top cardinality and pool,
    so that the load per register matches the full-size trace.  Returns
    (X, n_plain, exact cardinality) of every host after the window of the last
    k slices is complete."""
    from synth import traffic
    import oracle
    from oracle import exact
    k = 30
    slices = slices or k + 1
    gen = traffic.ZipfTraffic(1_000_000 // scale, 1.05, 2_000_000 // scale, k, seed=seed,
                              repeat_frac=0.10)
    o = oracle.Oracle("gfast", k=k, Z=(1 << 24) // scale, b=8, seed=0x9E3779B97F4A7C15)
    hist = []
    for _ in range(slices):
        s = gen.next_slice((64 << 20) // scale)
        hist.append(s)
        o.scan(s)
        o.slide()
    truth = exact.window_cardinalities(hist, slices - 1, k, gen.aips)
    X, n_plain = o.features(gen.aips)
    live = truth > 0
    return X[live], n_plain[live], truth[live].astype(np.float64)


def training_set(seeds, scale: int = 16, processes: int = 1):
    """Concatenated trace_shaped_run outputs of several seeds."""
    if processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            parts = pool.starmap(trace_shaped_run, [(s, scale) for s in seeds])
    else:
        parts = [trace_shaped_run(s, scale) for s in seeds]
    X = np.concatenate([p[0] for p in parts])
    n_plain = np.concatenate([p[1] for p in parts])
    card = np.concatenate([p[2] for p in parts])
    return X, n_plain, card
