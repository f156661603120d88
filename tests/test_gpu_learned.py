"""GPU tests of the learned augmentation (rcg_learn_*), against the oracle's
network (oracle/cnn.py) on the same seeded weights and inputs.

* forward pass: bfloat16 (inference) and float32 (training) weights, outputs
  within float32 rounding of the float64 oracle;
* gradient: the loss and its gradient with respect to the master weights
  against the oracle's loss and central finite differences of it;
* features and x_hat: coarse features equal the oracle's up to isolated
  one-ulp bfloat16 rounding flips (float32 vs float64 block means), x_hat the
  oracle's upsampling of the network output;
* the solver with the augmentation: pairs are recorded, training lowers the
  loss, and every solve still meets its tolerance by the oracle's residual,
  with the learned column accepted into U_j.
"""
import numpy as np
import pytest

from oracle import cnn, operator as op
from synthetic.cnn_init import init_weights
from tests.gpu_common import oracle_seed_inputs, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rcg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1602_00138_gb300 import rcg as r
    return r


def _weights(seed):
    th = init_weights(seed).astype(np.float64)
    rng = np.random.default_rng(50 + seed)
    # non-zero biases so that they are exercised
    o = 0
    for ci, co in zip(cnn.CHANNELS[:-1], cnn.CHANNELS[1:]):
        o += co * ci * 27
        th[o:o + co] = 0.05 * rng.standard_normal(co)
        o += co
    return th.astype(np.float32)


def _ctx(rcg, name, **opts):
    inp = workload(name)
    wl = inp["wl"]
    ctx = rcg.Context(wl.dim, wl.N, wl.robin_A, precision=rcg.RCG_MIXED, order=rcg.RCG_WAVE, k_u=wl.k_u,
                      keep_solutions=1, **opts)
    ctx.set_diffusion(inp["D"])
    ctx.set_sources_detectors(inp["src_ij"], inp["det_ij"])
    ctx.set_tolerances(inp["tol"])
    for s in range(wl.K + 1):
        ctx.set_sample(s, inp["mu"][s])
    return inp, ctx


def test_forward_matches_oracle(rcg):
    inp, ctx = _ctx(rcg, "t3d_32")
    try:
        Gx, Gy, Gz, f = ctx.learn_geometry()
        assert (Gx, Gy, Gz, f) == (8, 8, 8, 4)
        theta = _weights(1)
        ctx.learn_set_weights(theta)
        rng = np.random.default_rng(11)
        x = cnn.bf16(rng.standard_normal((3, 2, Gz, Gy, Gx)))
        for rounded in (True, False):
            out = ctx.learn_forward(x, rounded=rounded)
            for b in range(3):
                ref = cnn.forward(theta, x[b], round_weights=rounded)
                err = np.max(np.abs(out[b] - ref)) / np.max(np.abs(ref))
                assert err < 2e-5, (rounded, b, err)
        assert np.array_equal(ctx.learn_get_weights(), theta)
    finally:
        ctx.close()


def test_gradient_matches_finite_differences_of_the_oracle_loss(rcg):
    inp, ctx = _ctx(rcg, "t3d_16")
    try:
        Gx, Gy, Gz, f = ctx.learn_geometry()
        theta = _weights(2)
        ctx.learn_set_weights(theta)
        rng = np.random.default_rng(12)
        x = cnn.bf16(rng.standard_normal((2, 2, Gz, Gy, Gx)))
        t = rng.standard_normal((2, Gz, Gy, Gx))
        loss, g = ctx.learn_gradient(x, t)
        th64 = theta.astype(np.float64)
        ref_loss = cnn.loss(th64, list(x), list(t))
        assert abs(loss - ref_loss) <= 1e-5 * ref_loss
        P = cnn.n_params()
        idx = np.unique(np.concatenate([rng.integers(0, P, 40), [P - 1, P - 2, 864, 880]]))
        gmax = np.max(np.abs(g))
        for i in idx:
            h = 1e-4 * max(1.0, abs(th64[i]))
            tp, tm = th64.copy(), th64.copy()
            tp[i] += h
            tm[i] -= h
            fd = (cnn.loss(tp, list(x), list(t)) - cnn.loss(tm, list(x), list(t))) / (2 * h)
            assert abs(g[i] - fd) <= 2e-3 * gmax + 1e-3 * abs(fd), (i, g[i], fd)
    finally:
        ctx.close()


def test_features_and_prediction_match_oracle(rcg):
    inp, ctx = _ctx(rcg, "t3d_32")
    try:
        wl = inp["wl"]
        theta = _weights(3)
        ctx.learn_set_weights(theta)
        dims = (wl.N, wl.N, wl.N)
        f = cnn.pool_factor(dims)
        rng = np.random.default_rng(13)
        r0 = rng.standard_normal(wl.N ** 3).astype(np.float32)
        s = 2
        feat, xhat = ctx.learn_predict(s, r0)
        ref = cnn.features(r0.astype(np.float64), inp["mu"][s], dims, f)
        diff = np.abs(feat - ref)
        # isolated bfloat16 rounding flips only: one ulp (2^-8 relative) at most, on few entries
        assert np.all(diff <= 2.0 ** -7 * np.abs(ref) + 1e-30)
        assert np.count_nonzero(diff) <= max(2, feat.size // 500)
        out = cnn.forward(theta, feat.astype(np.float64))
        ref_x = cnn.upsample(out, dims, f)
        assert np.max(np.abs(xhat - ref_x)) <= 2e-5 * np.max(np.abs(ref_x))
    finally:
        ctx.close()


def test_learned_solves_meet_tolerance_and_training_lowers_the_loss(rcg):
    inp, ctx = _ctx(rcg, "t3d_32", learned=1, tau_rank=1e-6)
    try:
        wl = inp["wl"]
        U0, As, Bt, Ct = oracle_seed_inputs("t3d_32")
        ctx.learn_set_weights(init_weights(0))
        ctx.learn_record(True)
        ctx.seed(0, U0)
        stats, rc = ctx.solve_all(1, wl.K)
        assert rc == 0
        ncg = sum(1 for s_ in stats if s_["iters"] > 0)
        assert ctx.learn_pairs() == ncg > 0
        first = ctx.learn_train(1, batch=8, lr=1e-3, seed=1)
        last = ctx.learn_train(40, batch=8, lr=1e-3, seed=2)
        assert last < first
        ctx.learn_record(False)
        ctx.reset_to_seed()
        stats, rc = ctx.solve_all(1, wl.K)
        assert rc == 0
        B = np.hstack([Bt, Ct])
        aug = 0
        for s_ in stats:
            i, j = s_["sample"], s_["rhs"]
            x = ctx.solutions(i)[:, j]
            res = np.linalg.norm(B[:, j] - As[i] @ x) / np.linalg.norm(B[:, j])
            assert res <= inp["tol"][j] * 1.0000001, (i, j, res)
            aug += s_["augmented"]
        assert aug > 0 and aug <= ncg + 5
    finally:
        ctx.close()
