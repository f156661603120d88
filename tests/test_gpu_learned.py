"""GPU tests of the learned augmentation (rcg_learn_*): the U-Net on the
tensor cores against the oracle's network (oracle/cnn.py) on the same seeded
weights and inputs.

* forward pass (inference: bfloat16 weights and activations, float32 sums on
  the tensor cores) against the oracle's inference network (the same
  bfloat16 roundings, float64 sums): the sums differ in rounding only, which
  can flip an activation's bfloat16 rounding by one ulp (2^-8 relative) on
  isolated nodes, and the later layers spread each flip over their receptive
  field (measured: at most 7e-3 of the largest output magnitude, 9e-4 in the
  mean on a 21^3 coarse grid); the outputs must agree to 2e-2 and 3e-3 (an
  indexing or layout fault gives errors of order one), on grids with whole
  and ragged tiles, odd level dims and a 2D grid;
* gradient: the loss and its gradient with respect to the master weights
  (the training pass, bfloat16 operands) against the oracle's exact loss and
  central finite differences of it, to bfloat16 precision;
* features and x_hat: coarse features equal the oracle's up to isolated
  one-ulp bfloat16 rounding flips (float32 vs float64 block means), x_hat the
  oracle's upsampling of the oracle network's output on those features;
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
    for ci, co in cnn.LAYERS:
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


def _forward_errors(out, ref):
    """Largest and mean absolute difference relative to max|ref|."""
    sc = np.max(np.abs(ref))
    d = np.abs(out - ref)
    return np.max(d) / sc, np.mean(d) / sc


@pytest.mark.parametrize("name,geom", [("t3d_32", (8, 8, 8, 4)), ("t3d_21", (21, 21, 21, 1)),
                                       ("t2d_37", (37, 1, 37, 1))])
def test_forward_matches_oracle(rcg, name, geom):
    inp, ctx = _ctx(rcg, name)
    try:
        Gx, Gy, Gz, f = ctx.learn_geometry()
        assert (Gx, Gy, Gz, f) == geom
        theta = _weights(1)
        ctx.learn_set_weights(theta)
        rng = np.random.default_rng(11)
        x = cnn.bf16(rng.standard_normal((3, 2, Gz, Gy, Gx)))
        out = ctx.learn_forward(x)
        for b in range(3):
            ref = cnn.forward(theta, x[b])
            emax, emean = _forward_errors(out[b], ref)
            print(name, b, emax, emean)
            assert emax < 2e-2 and emean < 3e-3, (name, b, emax, emean)
        assert np.array_equal(ctx.learn_get_weights(), theta)
    finally:
        ctx.close()


def _layer_offsets():
    o, out = 0, []
    for ci, co in cnn.LAYERS:
        out.append((o, o + co * ci * 27))      # weights, biases
        o += co * ci * 27 + co
    return out


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
        # the training pass computes with bfloat16 operands: its loss is the
        # exact network's to bfloat16 precision
        assert abs(loss - ref_loss) <= 2e-2 * ref_loss, (loss, ref_loss)
        P = cnn.n_params()
        # random entries plus, per layer, a weight and a bias; the skip parts
        # of the stacked inputs of layers 5 and 7; the two real input channels of layer 0
        offs = _layer_offsets()
        picks = [rng.integers(0, P, 24)]
        for l, (wo, bo) in enumerate(offs):
            picks.append([wo + rng.integers(0, bo - wo), bo])
        ci5, ci7 = cnn.LAYERS[5][0], cnn.LAYERS[7][0]
        picks.append([offs[5][0] + (3 * ci5 + 70) * 27 + 13, offs[7][0] + (2 * ci7 + 40) * 27 + 4])
        picks.append([offs[0][0] + (5 * 2 + 1) * 27 + 22, P - 1])
        idx = np.unique(np.concatenate(picks))
        gmax = np.max(np.abs(g))
        fds = []
        for i in idx:
            h = 1e-4 * max(1.0, abs(th64[i]))
            tp, tm = th64.copy(), th64.copy()
            tp[i] += h
            tm[i] -= h
            fds.append((cnn.loss(tp, list(x), list(t)) - cnn.loss(tm, list(x), list(t))) / (2 * h))
        fds = np.array(fds)
        gi = g[idx].astype(np.float64)
        err = np.abs(gi - fds)
        print("gradient: max err / gmax", np.max(err) / gmax, "cos", gi @ fds / np.linalg.norm(gi) / np.linalg.norm(fds))
        assert np.all(err <= 3e-2 * gmax + 3e-2 * np.abs(fds)), list(zip(idx, gi, fds))
        assert gi @ fds >= 0.995 * np.linalg.norm(gi) * np.linalg.norm(fds)
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
        emax, emean = _forward_errors(xhat, ref_x)
        assert emax < 2e-2 and emean < 3e-3, (emax, emean)
    finally:
        ctx.close()


@pytest.mark.parametrize("mode", ["deflate", "start"])
def test_learned_solves_meet_tolerance_and_training_lowers_the_loss(rcg, mode):
    lm = rcg.RCG_LEARN_START if mode == "start" else rcg.RCG_LEARN_DEFLATE
    inp, ctx = _ctx(rcg, "t3d_32", learned=1, tau_rank=1e-6, learned_mode=lm)
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
