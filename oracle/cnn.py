"""Learned augmentation of the private recycle space (float64 restatement).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Not in the paper: the learned step of the build's contender.  For a
right-hand side j at sample i whose Galerkin check failed, a small 3D CNN
maps its check residual r0_j and the absorption mu_i to the coarse shape of
the correction g_j = A~_i^-1 r0_j that the inner deflated CG (eq. resi) must
find; the upsampled prediction x_hat joins the private U_j of that solve only
(never V) unless its Galerkin pivot is below tau_rank.  The network works on
a coarse grid (block means over f^3 fine nodes), which gives it a receptive
field of most of the domain at a small cost.

Definitions (all float64 here; the product computes in float32 from the same
bfloat16-rounded weights and inputs):

  f            pooling factor: 4 if every pooled axis is divisible by 4,
               else 2, else 1 (the y axis of a 2D grid, Ny = 1, is kept)
  coarse(v)    mean of v over each f x f x f block            (pool)
  input        [ coarse(r0) / max|coarse(r0)| ,
                 coarse(mu) / mean(mu) - 1 ], rounded to bfloat16
  h_0 = input; h_{l+1} = relu(conv_l(h_l)) for l < L-1; out = conv_{L-1}(h_{L-1})
  conv(h)[co, z, y, x] = b[co] + sum_ci sum_{dz,dy,dx in -1..1}
                         W[co, ci, dz+1, dy+1, dx+1] h[ci, z+dz, y+dy, x+dx]
               (zero outside the coarse grid; weights rounded to bfloat16)
  x_hat        trilinear interpolation of out from coarse cell centres to the
               fine nodes, clamped at the ends                 (upsample)
  target       coarse(g) / max|coarse(g)|
  loss         mean over pairs and coarse nodes of (out - target)^2, with the
               unrounded (float32 master) weights of training

Parameter vector layout (shared with the C ABI): for each layer l in order,
W_l [Cout][Cin][27] (offset index (dz+1)*9 + (dy+1)*3 + (dx+1)) then b_l
[Cout]; channels CHANNELS = (2, 16, 16, 16, 16, 16, 1).

Arrays are [channel][z][y][x] (x fastest), the node order of the grid.
Parity: pinned by tests/test_oracle_cnn.py (scipy correlation for the
convolution, torch's bfloat16 conversion for the rounding, exactness of the
interpolation on linear fields, block means by explicit loops).
"""
from __future__ import annotations

import numpy as np

CHANNELS = (2, 16, 16, 16, 16, 16, 1)


def n_params(channels=CHANNELS):
    return sum(co * ci * 27 + co for ci, co in zip(channels[:-1], channels[1:]))


def split_params(theta, channels=CHANNELS):
    """Flat parameter vector -> list of (W [Cout, Cin, 3, 3, 3], b [Cout])."""
    out, o = [], 0
    for ci, co in zip(channels[:-1], channels[1:]):
        W = np.asarray(theta[o:o + co * ci * 27], dtype=np.float64).reshape(co, ci, 3, 3, 3)
        o += co * ci * 27
        b = np.asarray(theta[o:o + co], dtype=np.float64)
        o += co
        out.append((W, b))
    assert o == len(theta)
    return out


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)


def pool_factor(dims):
    """dims = (Nx, Ny, Nz); Ny == 1 (2D) is never pooled."""
    axes = [d for d in dims if d > 1]
    for f in (4, 2):
        if all(d % f == 0 for d in axes):
            return f
    return 1


def coarse_dims(dims, f):
    Nx, Ny, Nz = dims
    return (Nx // f, Ny // f if Ny > 1 else 1, Nz // f)


def pool(v, dims, f):
    """Block means of a fine node vector -> coarse array [Gz, Gy, Gx]."""
    Nx, Ny, Nz = dims
    fy = f if Ny > 1 else 1
    a = np.asarray(v, dtype=np.float64).reshape(Nz, Ny, Nx)
    Gx, Gy, Gz = coarse_dims(dims, f)
    return a.reshape(Gz, f, Gy, fy, Gx, f).mean(axis=(1, 3, 5))


def features(r0, mu, dims, f):
    """The two bfloat16 input channels of a (residual, sample) pair."""
    cr = pool(r0, dims, f)
    cm = pool(mu, dims, f)
    a = np.max(np.abs(cr))
    ch0 = cr / a if a > 0 else cr
    ch1 = cm / np.mean(np.asarray(mu, dtype=np.float64)) - 1.0
    return bf16(np.stack([ch0, ch1]))


def target(g, dims, f):
    c = pool(g, dims, f)
    a = np.max(np.abs(c))
    return c / a if a > 0 else c


def conv3(h, W, b):
    """Zero-padded 3x3x3 correlation with bias: h [Cin, Gz, Gy, Gx]."""
    Cin, Gz, Gy, Gx = h.shape
    Cout = W.shape[0]
    hp = np.zeros((Cin, Gz + 2, Gy + 2, Gx + 2))
    hp[:, 1:-1, 1:-1, 1:-1] = h
    out = np.empty((Cout, Gz, Gy, Gx))
    for co in range(Cout):
        acc = np.full((Gz, Gy, Gx), b[co], dtype=np.float64)
        for dz in range(3):
            for dy in range(3):
                for dx in range(3):
                    win = hp[:, dz:dz + Gz, dy:dy + Gy, dx:dx + Gx]
                    acc += np.tensordot(W[co, :, dz, dy, dx], win, axes=(0, 0))
        out[co] = acc
    return out


def forward(theta, inp, channels=CHANNELS, round_weights=True):
    """Network output [Gz, Gy, Gx] for one input [2, Gz, Gy, Gx]; inference
    rounds the weights to bfloat16, training (round_weights=False) uses them
    as given (the float32 master copy)."""
    layers = split_params(bf16(theta) if round_weights else np.asarray(theta, dtype=np.float64), channels)
    h = np.asarray(inp, dtype=np.float64)
    for l, (W, b) in enumerate(layers):
        h = conv3(h, W, b)
        if l < len(layers) - 1:
            h = np.maximum(h, 0.0)
    return h[0]


def _interp_axis(c, n_fine, f, axis):
    G = c.shape[axis]
    if G == 1 or f == 1:
        return np.repeat(c, n_fine // G, axis=axis) if G != n_fine else c
    t = (np.arange(n_fine) + 0.5) / f - 0.5
    i0 = np.floor(t).astype(int)
    w = t - i0
    lo = np.clip(i0, 0, G - 1)
    hi = np.clip(i0 + 1, 0, G - 1)
    shape = [1] * c.ndim
    shape[axis] = n_fine
    w = w.reshape(shape)
    return np.take(c, lo, axis=axis) * (1 - w) + np.take(c, hi, axis=axis) * w


def upsample(out, dims, f):
    """Trilinear interpolation of a coarse array to the fine node vector."""
    Nx, Ny, Nz = dims
    a = _interp_axis(out, Nx, f, 2)
    a = _interp_axis(a, Ny, f if Ny > 1 else 1, 1)
    a = _interp_axis(a, Nz, f, 0)
    return a.reshape(-1)


def predict(theta, r0, mu, dims, channels=CHANNELS):
    """x_hat on the fine grid for one right-hand side."""
    f = pool_factor(dims)
    return upsample(forward(theta, features(r0, mu, dims, f), channels), dims, f)


def loss(theta, inputs, targets, channels=CHANNELS):
    """Training loss: mean squared error over pairs and coarse nodes, with the
    unrounded (master) weights."""
    tot, cnt = 0.0, 0
    for inp, t in zip(inputs, targets):
        d = forward(theta, inp, channels, round_weights=False) - t
        tot += float(np.sum(d * d))
        cnt += d.size
    return tot / cnt
