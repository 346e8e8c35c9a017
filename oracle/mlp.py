"""Plain FP64 reference of the network that guesses the inversion's starting
point (test infrastructure only; the CUDA library never imports it).

The network (no counterpart in the paper, which starts Newton from the
previous primitives, Sec. 2.6) maps the ten inputs of `ora_mlp_features`
to the two targets of `ora_mlp_targets`:

    x  = (f - fmean) / fstd                        standardised inputs (10)
    h1 = tanh(W1 x  + b1)                          64
    h2 = tanh(W2 h1 + b2)                          64
    h3 = tanh(W3 h2 + b3)                          64
    yn = W4 h3 + b4                                2, standardised
    y  = yn * ystd + ymean

Parameters travel as one flat vector in the order W1 (64 x 10, row = output
unit), b1, W2 (64 x 64), b2, W3, b3, W4 (2 x 64), b4 -- 9154 values -- and
the standardisation as (fmean[10], fstd[10], ymean[2], ystd[2]).

Training loss: mean over samples and both outputs of (yn - (t - ymean)/ystd)^2.

`forward(..., bf16=True)` states what the tensor-core inference computes:
the standardised input and the hidden activations h1, h2 that feed a matrix
product are rounded to bfloat16 (round to nearest, ties to even), as are
W1..W4; products accumulate in FP32 (here: exactly, in FP64); biases and
tanh stay FP32 (FP64 here); the output layer takes h3 unrounded.
"""
import numpy as np

SIZES = (10, 64, 64, 64, 2)
SHAPES = [(64, 10), (64,), (64, 64), (64,), (64, 64), (64,), (2, 64), (2,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)  # 9154
N_NORM = 24


def unpack(theta):
    """Flat parameter vector -> [W1, b1, W2, b2, W3, b3, W4, b4] (views, FP64)."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def split_norm(norm):
    norm = np.asarray(norm, dtype=np.float64)
    return norm[0:10], norm[10:20], norm[20:22], norm[22:24]


def bf16_round(x):
    """Round FP32 values to the nearest bfloat16 (ties to even); returned as float64.

    bfloat16 keeps the top 16 bits of an IEEE binary32: adding 0x7FFF plus the
    lowest kept bit before truncating rounds to nearest with ties to even."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    r = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


def forward(theta, norm, F, bf16=False, hidden=False):
    """F: (n, 10) inputs -> (n, 2) outputs in target units (and the hidden layers if asked)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    fm, fs, ym, ys = split_norm(norm)
    x = (np.asarray(F, dtype=np.float64) - fm) / fs
    if bf16:
        W1, W2, W3, W4 = (bf16_round(w) for w in (W1, W2, W3, W4))
        x = bf16_round(x)
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh((bf16_round(h1) if bf16 else h1) @ W2.T + b2)
    h3 = np.tanh((bf16_round(h2) if bf16 else h2) @ W3.T + b3)
    yn = h3 @ W4.T + b4
    y = yn * ys + ym
    return (y, (x, h1, h2, h3, yn)) if hidden else y


def loss_and_grad(theta, norm, F, T):
    """Mean squared error of the standardised outputs and its gradient (9154) by backpropagation."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    fm, fs, ym, ys = split_norm(norm)
    _, (x, h1, h2, h3, yn) = forward(theta, norm, F, hidden=True)
    tn = (np.asarray(T, dtype=np.float64) - ym) / ys
    n = x.shape[0]
    r = yn - tn
    loss = float((r * r).sum() / (2 * n))
    dyn = r * (2.0 / (2 * n))                    # dL/dyn
    gW4 = dyn.T @ h3
    gb4 = dyn.sum(axis=0)
    dz3 = (dyn @ W4) * (1.0 - h3 * h3)
    gW3 = dz3.T @ h2
    gb3 = dz3.sum(axis=0)
    dz2 = (dz3 @ W3) * (1.0 - h2 * h2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(axis=0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4])


def loss(theta, norm, F, T):
    fm, fs, ym, ys = split_norm(norm)
    y = forward(theta, norm, F)
    r = (y - np.asarray(T, dtype=np.float64)) / ys
    return float((r * r).mean())
