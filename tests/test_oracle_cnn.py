"""Pins of the oracle's learned-augmentation network (oracle/cnn.py) against
facts independent of its own formulas: scipy's correlation, torch's bfloat16
conversion, block means by explicit loops, exactness of linear interpolation,
and special networks with a known output."""
import numpy as np
import pytest
import scipy.signal

from oracle import cnn


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(5000).astype(np.float32) * 10.0 ** rng.integers(-6, 6, 5000),
                        np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 0.0,
                                  65504.0, 1e-30], dtype=np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(cnn.bf16(x), ref)
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert cnn.bf16(np.float32(1.0 + 2.0 ** -8)) == 1.0


def test_conv3_matches_scipy_correlation():
    rng = np.random.default_rng(4)
    h = rng.standard_normal((3, 5, 4, 6))
    W = rng.standard_normal((2, 3, 3, 3, 3))
    b = rng.standard_normal(2)
    out = cnn.conv3(h, W, b)
    for co in range(2):
        ref = b[co] + sum(scipy.signal.correlate(h[ci], W[co, ci], mode="same") for ci in range(3))
        assert np.allclose(out[co], ref, rtol=1e-13, atol=1e-13)


def test_conv3_on_a_one_cell_thick_axis_is_a_2d_correlation():
    rng = np.random.default_rng(5)
    h = rng.standard_normal((2, 6, 1, 7))
    W = rng.standard_normal((1, 2, 3, 3, 3))
    out = cnn.conv3(h, W, np.zeros(1))
    ref = sum(scipy.signal.correlate(h[ci, :, 0, :], W[0, ci, :, 1, :], mode="same") for ci in range(2))
    assert np.allclose(out[0, :, 0, :], ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dims,f", [((8, 4, 8), 2), ((8, 8, 12), 4), ((12, 1, 8), 4)])
def test_pool_is_the_block_mean(dims, f):
    rng = np.random.default_rng(6)
    Nx, Ny, Nz = dims
    v = rng.standard_normal(Nx * Ny * Nz)
    c = cnn.pool(v, dims, f)
    Gx, Gy, Gz = cnn.coarse_dims(dims, f)
    fy = f if Ny > 1 else 1
    for kz in range(Gz):
        for ky in range(Gy):
            for kx in range(Gx):
                s, cnt = 0.0, 0
                for z in range(kz * f, kz * f + f):
                    for y in range(ky * fy, ky * fy + fy):
                        for x in range(kx * f, kx * f + f):
                            s += v[x + Nx * (y + Ny * z)]
                            cnt += 1
                assert abs(c[kz, ky, kx] - s / cnt) < 1e-14


def test_pool_factor():
    assert cnn.pool_factor((64, 64, 64)) == 4
    assert cnn.pool_factor((64, 1, 64)) == 4
    assert cnn.pool_factor((6, 6, 10)) == 2
    assert cnn.pool_factor((21, 21, 21)) == 1


def test_upsample_reproduces_constants_and_linear_fields():
    dims, f = (16, 8, 12), 4
    Gx, Gy, Gz = cnn.coarse_dims(dims, f)
    up = cnn.upsample(np.full((Gz, Gy, Gx), 2.5), dims, f)
    assert np.allclose(up, 2.5, rtol=0, atol=1e-15)
    # linear in the coarse x index: exact at fine nodes whose coordinate lies
    # between the first and last coarse centres, clamped outside
    c = np.broadcast_to((1.0 + 0.5 * np.arange(Gx))[None, None, :], (Gz, Gy, Gx)).copy()
    up = cnn.upsample(c, dims, f).reshape(dims[2], dims[1], dims[0])
    t = (np.arange(dims[0]) + 0.5) / f - 0.5
    expect = 1.0 + 0.5 * np.clip(t, 0, Gx - 1)
    assert np.allclose(up[3, 2, :], expect, rtol=0, atol=1e-14)


def test_identity_network_returns_its_input():
    channels = (1, 1)
    theta = np.zeros(cnn.n_params(channels))
    theta[13] = 1.0                       # W[0, 0, 1, 1, 1]: the centre tap
    inp = np.random.default_rng(7).standard_normal((1, 3, 4, 5))
    assert np.array_equal(cnn.forward(theta, inp, channels), inp[0])


def test_relu_between_layers_and_linear_last_layer():
    channels = (1, 1, 1)
    theta = np.zeros(cnn.n_params(channels))
    theta[13] = 1.0                       # layer 0: identity, then ReLU
    theta[28 + 13] = -2.0                 # layer 1 (offset 27 + 1 bias): -2 x, no ReLU
    inp = np.random.default_rng(8).standard_normal((1, 2, 3, 4))
    assert np.allclose(cnn.forward(theta, inp, channels), -2.0 * np.maximum(inp[0], 0.0))


def test_features_are_normalised():
    dims = (16, 16, 16)
    rng = np.random.default_rng(9)
    r0 = rng.standard_normal(16 ** 3)
    mu = 0.01 + 0.02 * rng.random(16 ** 3)
    x = cnn.features(r0, mu, dims, 4)
    assert x.shape == (2, 4, 4, 4)
    assert abs(np.max(np.abs(x[0])) - 1.0) < 2 ** -8
    assert abs(np.mean(x[1])) < 2 ** -7           # block means average to the global mean
    assert cnn.n_params() == 29025


def test_target_is_the_block_mean_over_its_largest_magnitude():
    """Hand-computed: two coarse cells (f = 4 on a 4 x 4 x 8 grid) whose fine
    values alternate 1, 3 (block mean 2) and -2, -6 (block mean -4); the
    target divides the block means by the largest |block mean|, 4, and not by
    the largest fine value (6) or a sum."""
    dims = (4, 4, 8)
    g = np.empty(4 * 4 * 8)
    for z in range(8):
        for y in range(4):
            for x in range(4):
                odd = (x + y + z) % 2
                g[x + 4 * (y + 4 * z)] = (3.0 if odd else 1.0) if z < 4 else (-6.0 if odd else -2.0)
    t = cnn.target(g, dims, cnn.pool_factor(dims))
    assert t.shape == (2, 1, 1)
    assert t[0, 0, 0] == 0.5 and t[1, 0, 0] == -1.0


def test_loss_is_the_mean_over_pairs_and_coarse_nodes_with_master_weights():
    """Hand-computed on a one-layer network (only the centre tap w and the
    bias b set) and two 2 x 2 x 2 pairs: pair 1 has input 1 and target 1.5
    everywhere, pair 2 input 0 and target 0 except 2.5 at one node.  With
    w = 2 + 2^-10 (not a bfloat16 value: the loss must use it unrounded) and
    b = 0.5 the squared errors sum to 8 (1 + 2^-10)^2 over pair 1 and
    7 * 0.25 + 4 over pair 2; the loss is their total over 16 nodes (a sum,
    or a mean per pair only, would differ)."""
    channels = (1, 1)
    theta = np.zeros(cnn.n_params(channels))
    w = 2.0 + 2.0 ** -10
    theta[13] = w
    theta[27] = 0.5
    inputs = [np.ones((1, 2, 2, 2)), np.zeros((1, 2, 2, 2))]
    t2 = np.zeros((2, 2, 2))
    t2[1, 0, 1] = 2.5
    targets = [np.full((2, 2, 2), 1.5), t2]
    expect = (8 * (1.0 + 2.0 ** -10) ** 2 + 7 * 0.25 + 4.0) / 16
    assert abs(cnn.loss(theta, inputs, targets, channels) - expect) < 1e-15
    # the rounded weights (inference) would give a different value
    assert cnn.bf16(np.float32(w)) == 2.0
