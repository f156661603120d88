"""Learned augmentation of the private recycle space (float64 restatement).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Not in the paper: the learned step of the build's contender.  For a
right-hand side j at sample i whose Galerkin check failed, a 3D U-Net maps
its check residual r0_j and the absorption mu_i to the coarse shape of the
correction g_j = A~_i^-1 r0_j that the inner deflated CG (eq. resi) must
find; the upsampled prediction x_hat joins the private U_j of that solve only
(never V) unless its Galerkin pivot is below tau_rank.  The network works on
a coarse grid (block means over f^3 fine nodes) and halves it twice more
inside, which gives it a receptive field of the whole domain.

Definitions (float64 here; the product computes with bfloat16 operands and
float32 sums at the rounding points marked [r] below):

  f            pooling factor: 4 if every pooled axis is divisible by 4,
               else 2, else 1 (the y axis of a 2D grid, Ny = 1, is kept)
  coarse(v)    mean of v over each f x f x f block            (pool)
  input        [ coarse(r0) / max|coarse(r0)| ,
                 coarse(mu) / mean(mu) - 1 ], rounded to bfloat16
  conv(h; l)   zero-padded 3x3x3 correlation with bias:
               conv(h)[co, z, y, x] = b[co] + sum_ci sum_{dz,dy,dx in -1..1}
                                      W[co, ci, dz+1, dy+1, dx+1] h[ci, z+dz, y+dy, x+dx]
  R(h)         max(h, 0), then [r] rounded to bfloat16
  down(h)      level halving: a cell of dims ceil(G / 2) per axis is the mean
               of the (up to 8) cells 2k, 2k+1 of each axis inside the grid,
               then [r] rounded to bfloat16
  up(h, G)     nearest-cell doubling to dims G: up(h)[z, y, x] = h[z//2, y//2, x//2]
  network      (levels 0, 1, 2 = the coarse grid, once and twice halved)
                 a0 = R(conv(input; 0))          16 channels, level 0
                 s0 = R(conv(a0; 1))             16, level 0 (skip)
                 a1 = R(conv(down(s0); 2))       32, level 1
                 s1 = R(conv(a1; 3))             32, level 1 (skip)
                 a2 = R(conv(down(s1); 4))       64, level 2
                 a3 = R(conv([up(a2), s1]; 5))   32, level 1 (96 input channels)
                 a4 = R(conv(a3; 6))             32, level 1
                 a5 = R(conv([up(a4), s0]; 7))   16, level 0 (48 input channels)
                 a6 = R(conv(a5; 8))             16, level 0
                 out = conv(a6; 9)               1 channel, level 0 (no ReLU)
               [a, b] stacks channels, a first.  Inference uses the
               bfloat16-rounded weights and all [r] roundings; the exact
               network (training's reference) uses neither.
  x_hat        trilinear interpolation of out from coarse cell centres to the
               fine nodes, clamped at the ends                 (upsample)
  target       coarse(g) / max|coarse(g)|
  loss         mean over pairs and coarse nodes of (out - target)^2 with the
               exact network at the (float32 master) weights

Parameter vector layout (shared with the C ABI): for each layer l = 0..9 in
order, W_l [Cout][Cin][27] (offset index (dz+1)*9 + (dy+1)*3 + (dx+1)) then
b_l [Cout], with (Cin, Cout) = LAYERS[l]: 243,473 parameters.

Arrays are [channel][z][y][x] (x fastest), the node order of the grid.
Parity: pinned by tests/test_oracle_cnn.py (scipy correlation for the
convolution, torch's bfloat16 conversion for the rounding, block means and
the level halving by explicit loops, exactness of the interpolation on
linear fields, and weight sets for which the network is a known function:
the skip path, the deep path through both halvings, the rounding points).
"""
from __future__ import annotations

import numpy as np

LAYERS = ((2, 16), (16, 16), (16, 32), (32, 32), (32, 64), (96, 32), (32, 32), (48, 16), (16, 16), (16, 1))


def n_params(layers=LAYERS):
    return sum(co * ci * 27 + co for ci, co in layers)


def split_params(theta, layers=LAYERS):
    """Flat parameter vector -> list of (W [Cout, Cin, 3, 3, 3], b [Cout])."""
    out, o = [], 0
    for ci, co in layers:
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


def half_dims(G):
    """Dims of the next level: ceil(G / 2) per axis."""
    return tuple((g + 1) // 2 for g in G)


def down(h):
    """Level halving of h [C, Gz, Gy, Gx]: mean of the cells of each 2 x 2 x 2
    block that lie inside the grid (fewer at an odd end, one on a length-1 axis)."""
    C, Gz, Gy, Gx = h.shape
    Hz, Hy, Hx = half_dims((Gz, Gy, Gx))
    s = np.zeros((C, Hz, Hy, Hx))
    cnt = np.zeros((Hz, Hy, Hx))
    for dz in range(2):
        for dy in range(2):
            for dx in range(2):
                part = h[:, dz::2, dy::2, dx::2]
                _, pz, py, px = part.shape
                s[:, :pz, :py, :px] += part
                cnt[:pz, :py, :px] += 1
    return s / cnt


def up(h, G):
    """Nearest-cell doubling of h [C, Hz, Hy, Hx] to dims G = (Gz, Gy, Gx)."""
    Gz, Gy, Gx = G
    iz, iy, ix = np.arange(Gz) // 2, np.arange(Gy) // 2, np.arange(Gx) // 2
    return h[:, iz][:, :, iy][:, :, :, ix]


def forward(theta, inp, exact=False, layers=LAYERS):
    """U-Net output [Gz, Gy, Gx] for one input [2, Gz, Gy, Gx].  Inference
    (exact=False) rounds the weights and every ReLU and halving output to
    bfloat16; exact=True (training's reference, the float32 master weights)
    rounds nothing."""
    P = split_params(np.asarray(theta, dtype=np.float64) if exact else bf16(theta), layers)
    rnd = (lambda a: a) if exact else bf16

    def R(h, l):
        return rnd(np.maximum(conv3(h, *P[l]), 0.0))

    x = np.asarray(inp, dtype=np.float64)
    G0 = x.shape[1:]
    a0 = R(x, 0)
    s0 = R(a0, 1)
    a1 = R(rnd(down(s0)), 2)
    G1 = a1.shape[1:]
    s1 = R(a1, 3)
    a2 = R(rnd(down(s1)), 4)
    a3 = R(np.concatenate([up(a2, G1), s1]), 5)
    a4 = R(a3, 6)
    a5 = R(np.concatenate([up(a4, G0), s0]), 7)
    a6 = R(a5, 8)
    return conv3(a6, *P[9])[0]


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


def predict(theta, r0, mu, dims):
    """x_hat on the fine grid for one right-hand side (inference)."""
    f = pool_factor(dims)
    return upsample(forward(theta, features(r0, mu, dims, f)), dims, f)


def loss(theta, inputs, targets):
    """Training loss: mean squared error over pairs and coarse nodes of the
    exact network at the given (master) weights."""
    tot, cnt = 0.0, 0
    for inp, t in zip(inputs, targets):
        d = forward(theta, inp, exact=True) - t
        tot += float(np.sum(d * d))
        cnt += d.size
    return tot / cnt
