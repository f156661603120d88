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


# offsets of the U-Net's layers in the parameter vector
def _offsets():
    w, o = [], 0
    for ci, co in cnn.LAYERS:
        w.append(o)
        o += co * ci * 27 + co
    return w


def _tap(theta, l, co, ci, val, tap=13):
    """W_l[co, ci] at one tap (13 = the centre) set to val."""
    ci_n = cnn.LAYERS[l][0]
    theta[_offsets()[l] + (co * ci_n + ci) * 27 + tap] = val


def _bias(theta, l, co, val):
    ci_n, co_n = cnn.LAYERS[l]
    theta[_offsets()[l] + co_n * ci_n * 27 + co] = val


def _skip_path(w9=1.0, b9=0.0):
    """Weights under which the U-Net is w9 relu(x0) + b9 through the level-0
    skip: conv 0, 1 copy channel 0, conv 7 takes the skip s0 (channel 32 of
    its input [up(a4), s0]), conv 8 copies, conv 9 scales; the deep path
    carries zeros."""
    th = np.zeros(cnn.n_params())
    _tap(th, 0, 0, 0, 1.0)
    _tap(th, 1, 0, 0, 1.0)
    _tap(th, 7, 0, 32, 1.0)
    _tap(th, 8, 0, 0, 1.0)
    _tap(th, 9, 0, 0, w9)
    _bias(th, 9, 0, b9)
    return th


def _deep_path():
    """Weights under which the U-Net is up(up(down(down(relu(x0))))) through
    both halvings: channel 0 copied by every conv, conv 5 takes up(a2)
    (channel 0 of [up(a2), s1]) and conv 7 takes up(a4) (channel 0 of
    [up(a4), s0])."""
    th = np.zeros(cnn.n_params())
    for l in range(10):
        _tap(th, l, 0, 0, 1.0)
    return th


def test_parameter_count_and_layer_table():
    # 3 levels, 16-32-64 channels, skip connections stacked after the upsampled path
    assert cnn.n_params() == 243473
    assert [ci for ci, _ in cnn.LAYERS] == [2, 16, 16, 32, 32, 96, 32, 48, 16, 16]
    assert [co for _, co in cnn.LAYERS] == [16, 16, 32, 32, 64, 32, 32, 16, 16, 1]


@pytest.mark.parametrize("dims", [(4, 6, 8), (5, 3, 7), (3, 1, 5)])
def test_down_is_the_mean_over_the_cells_inside_the_grid(dims):
    Gz, Gy, Gx = dims
    h = np.random.default_rng(12).standard_normal((2, Gz, Gy, Gx))
    d = cnn.down(h)
    assert d.shape == (2, (Gz + 1) // 2, (Gy + 1) // 2, (Gx + 1) // 2)
    for c in range(2):
        for kz in range(d.shape[1]):
            for ky in range(d.shape[2]):
                for kx in range(d.shape[3]):
                    vals = [h[c, z, y, x] for z in (2 * kz, 2 * kz + 1) for y in (2 * ky, 2 * ky + 1)
                            for x in (2 * kx, 2 * kx + 1) if z < Gz and y < Gy and x < Gx]
                    assert abs(d[c, kz, ky, kx] - sum(vals) / len(vals)) < 1e-15


def test_up_copies_the_parent_cell():
    h = np.random.default_rng(13).standard_normal((1, 2, 3, 2))
    u = cnn.up(h, (3, 5, 4))
    for z in range(3):
        for y in range(5):
            for x in range(4):
                assert u[0, z, y, x] == h[0, z // 2, y // 2, x // 2]


def test_skip_path_network_is_a_scaled_relu():
    inp = np.zeros((2, 4, 3, 5))
    inp[0] = np.random.default_rng(7).standard_normal((4, 3, 5))
    inp = cnn.bf16(inp)
    out = cnn.forward(_skip_path(-2.0, 0.25), inp, exact=True)
    assert np.array_equal(out, -2.0 * np.maximum(inp[0], 0.0) + 0.25)
    # inference rounds the weights: 2 + 2^-10 acts as 2
    out16 = cnn.forward(_skip_path(2.0 + 2.0 ** -10, 0.0), inp)
    assert np.array_equal(out16, 2.0 * np.maximum(inp[0], 0.0))


def test_deep_path_network_returns_block_constant_input():
    """On a grid of 4 x 4 x 4 blocks, a non-negative input constant on each
    block passes both halvings and doublings unchanged; a swapped stacking
    order of [up(.), skip] would return zeros here."""
    G = (8, 4, 12)
    blocks = np.random.default_rng(14).random((2, 1, 3))
    x0 = np.kron(blocks, np.ones((4, 4, 4)))
    inp = np.stack([x0, np.zeros(G)])
    assert np.allclose(cnn.forward(_deep_path(), inp, exact=True), x0, rtol=0, atol=1e-15)
    # odd dims: the explicit composition of the two halvings and doublings
    G = (5, 3, 7)
    x0 = np.random.default_rng(15).standard_normal(G)
    inp = np.stack([x0, np.zeros(G)])
    G1 = cnn.half_dims(G)
    ref = cnn.up(cnn.up(cnn.down(cnn.down(np.maximum(x0, 0.0)[None])), G1), G)[0]
    assert np.allclose(cnn.forward(_deep_path(), inp, exact=True), ref, rtol=0, atol=1e-15)


def test_inference_rounds_relu_outputs_and_halvings_to_bfloat16():
    # conv output (1 + 2^-7)^2 = 1 + 2^-6 + 2^-14 is rounded to 1 + 2^-6
    th = _skip_path()
    _tap(th, 0, 0, 0, 1.0 + 2.0 ** -7)
    inp = np.zeros((2, 2, 2, 2))
    inp[0] = 1.0 + 2.0 ** -7
    assert np.all(cnn.forward(th, inp) == 1.0 + 2.0 ** -6)
    assert np.all(cnn.forward(th, inp, exact=True) == 1.0 + 2.0 ** -6 + 2.0 ** -14)
    # a block mean 1 + 2^-10 is rounded to 1 by the halving
    inp = np.zeros((2, 2, 2, 2))
    inp[0] = 1.0
    inp[0, 1, 1, 1] = 1.0 + 2.0 ** -7
    assert np.all(cnn.forward(_deep_path(), inp) == 1.0)
    assert np.allclose(cnn.forward(_deep_path(), inp, exact=True), 1.0 + 2.0 ** -10, rtol=0, atol=1e-15)


def test_features_are_normalised():
    dims = (16, 16, 16)
    rng = np.random.default_rng(9)
    r0 = rng.standard_normal(16 ** 3)
    mu = 0.01 + 0.02 * rng.random(16 ** 3)
    x = cnn.features(r0, mu, dims, 4)
    assert x.shape == (2, 4, 4, 4)
    assert abs(np.max(np.abs(x[0])) - 1.0) < 2 ** -8
    assert abs(np.mean(x[1])) < 2 ** -7           # block means average to the global mean


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
    """Hand-computed with the skip-path weights (the network is
    w relu(x0) + b) on two 2 x 2 x 2 pairs: pair 1 has input 1 and target 1.5
    everywhere, pair 2 input 0 and target 0 except 2.5 at one node.  With
    w = 2 + 2^-10 (not a bfloat16 value: the loss must use it unrounded) and
    b = 0.5 the squared errors sum to 8 (1 + 2^-10)^2 over pair 1 and
    7 * 0.25 + 4 over pair 2; the loss is their total over 16 nodes (a sum,
    or a mean per pair only, would differ)."""
    w = 2.0 + 2.0 ** -10
    theta = _skip_path(w, 0.5)
    one = np.zeros((2, 2, 2, 2))
    one[0] = 1.0
    inputs = [one, np.zeros((2, 2, 2, 2))]
    t2 = np.zeros((2, 2, 2))
    t2[1, 0, 1] = 2.5
    targets = [np.full((2, 2, 2), 1.5), t2]
    expect = (8 * (1.0 + 2.0 ** -10) ** 2 + 7 * 0.25 + 4.0) / 16
    assert abs(cnn.loss(theta, inputs, targets) - expect) < 1e-15
    # the rounded weights (inference) would give a different value
    assert cnn.bf16(np.float32(w)) == 2.0
