"""Parity at the two large configurations, in the launch configurations the
bench times.

3D 128^3 (64 + 64 right-hand sides, 10 samples, tolerances 1e-8 / 1e-6
alternating; mixed precision, all 1280 lanes in one wave, V <= 1024):
  * every solve delivered (the library's float64 relres <= tol);
  * sampled delivered solutions within tolerance by the oracle's residual
    (scipy operator of that sample), both tolerance classes;
  * V orthonormal to float32 accuracy;
  * the reduced model and Jacobian at a sampled point equal the oracle's
    reduced model on the device basis (1e-6, the mixed acceptance tolerance);
  * Psi_r at samples 1 and 2 equals the plain float64 recycled-CG run's
    (same library, paper order, seeded from the contender) to 1e-6: both bases
    hold those samples' solutions to their tolerance, and the reduced transfer
    function's error is second order in it (Sec. 3.4).

3D 128^3 learned augmentation (64 + 64 right-hand sides, samples 1-2, tol
1e-8, learned + mixed in one wave; the U-Net trained on 512 plain-method
solves at four random 2-6-anomaly phantoms):
  * every solve delivered, sampled solutions within tolerance by the
    oracle's residual, the learned column accepted into U_j;
  * fewer mean CG iterations than mixed batched RCG without the network from
    the same seed;
  * Psi_r at samples 1 and 2 equals that run's to 1e-6.

3D 192^3 (128 + 128, samples 1-2 of 20, waves of one sample, V <= 2048):
  * every solve delivered; seed rank k_u + 256;
  * Psi_r at samples 1 and 2 equals the plain float64 run's to 1e-6 (the
    float64 run is itself checked against the oracle at the smaller sizes).
"""
import numpy as np
import pytest

from oracle import operator as op, rom
from synthetic.cnn_init import init_weights
from synthetic.phantom import make_workload, pals_mu, training_params

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


def _ctx(rcg, inp, K, **kw):
    wl = inp["wl"]
    ctx = rcg.Context(wl.dim, wl.N, wl.robin_A, k_u=wl.k_u, max_samples=K + 1, **kw)
    ctx.set_diffusion(inp["D"])
    ctx.set_sources_detectors(inp["src_ij"], inp["det_ij"])
    ctx.set_tolerances(inp["tol"])
    for s in range(K + 1):
        ctx.set_sample(s, inp["mu"][s])
    return ctx


def _fp64_psi(rcg, inp, contender, samples):
    """Psi_r at the given samples from the plain float64 run (paper order) over them."""
    ctx = _ctx(rcg, inp, max(samples), precision=rcg.RCG_FP64, order=rcg.RCG_SEQUENTIAL, tau_rank=1e-12,
               r_max=2048)
    try:
        ctx.seed_copy(contender)
        stats, rc = ctx.solve_all(1, max(samples))
        assert rc == 0
        return {s: ctx.rom_eval(inp["mu"][s])[0] for s in samples}
    finally:
        ctx.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_128_cubed_batched_wave(rcg):
    inp = make_workload("c3_3d128")
    wl = inp["wl"]
    ctx = _ctx(rcg, inp, wl.K, precision=rcg.RCG_MIXED, order=rcg.RCG_WAVE, tau_rank=1e-6, r_max=1024,
               keep_solutions=1)
    try:
        ctx.seed(0, None)
        stats, rc = ctx.solve_all(1, wl.K)
        assert rc == 0 and len(stats) == wl.K * wl.nrhs
        for s in stats:
            assert s["relres"] <= inp["tol"][s["rhs"]] * 1.0001, s
        # sampled solutions by the oracle's residual: both tolerance classes, sources and detectors
        for smp in (1, wl.K):
            A, Bt, Ct = op.assemble(inp, smp)
            B = np.hstack([Bt, Ct])
            X = ctx.solutions(smp)
            for j in (0, 1, wl.nsrc - 1, wl.nsrc, wl.nrhs - 2, wl.nrhs - 1):
                rr = np.linalg.norm(B[:, j] - A @ X[:, j]) / np.linalg.norm(B[:, j])
                assert rr <= inp["tol"][j] * 1.05, (smp, j, rr)
            del X
        V = ctx.basis()
        G = V.T @ V
        assert np.abs(G - np.eye(G.shape[0])).max() <= 5e-5
        # reduced model on the device basis at a sampled point (four parameters of the Jacobian)
        s = 3
        A, Bt, Ct = op.assemble(inp, s)
        dmu = inp["dmu"][s][:4]
        Pg, Jg = ctx.rom_eval(inp["mu"][s], dmu)
        Pv, Jv = rom.rom_eval(V, A, Bt, Ct, inp["h"], dmu)
        assert _rel(Pg, Pv) <= 1e-6, _rel(Pg, Pv)
        assert _rel(Jg, Jv) <= 1e-6, _rel(Jg, Jv)
        del V, A
        # against the plain float64 run over samples 1-2
        psi64 = _fp64_psi(rcg, inp, ctx, [1, 2])
        for smp, P in psi64.items():
            Pm = ctx.rom_eval(inp["mu"][smp])[0]
            assert _rel(Pm, P) <= 1e-6, (smp, _rel(Pm, P))
    finally:
        ctx.close()


def test_128_cubed_learned_augmentation(rcg):
    inp = make_workload("c4_3d128", K=2, with_dmu=False)
    wl = inp["wl"]
    ntrain = 4
    ctx = rcg.Context(wl.dim, wl.N, wl.robin_A, k_u=wl.k_u, max_samples=3 + ntrain, precision=rcg.RCG_MIXED,
                      order=rcg.RCG_WAVE, tau_rank=1e-6, r_max=1024, keep_solutions=1, learned=1)
    ctx.set_diffusion(inp["D"])
    ctx.set_sources_detectors(inp["src_ij"], inp["det_ij"])
    ctx.set_tolerances(inp["tol"])
    for s in range(3):
        ctx.set_sample(s, inp["mu"][s])
    plain = None
    try:
        X = np.asarray(inp["X"])
        grid = (wl.N, wl.h, wl.dim)
        for i, p in enumerate(training_params(wl, ntrain)):
            ctx.set_sample(3 + i, pals_mu(p, X, wl.mu_bg, grid))
        ctx.seed(0, None)
        ctx.learn_set_weights(init_weights(0))
        ctx.learn_record(True)
        stats, rc = ctx.solve_all(3, ntrain)
        assert rc == 0
        assert ctx.learn_pairs() == ntrain * wl.nrhs
        first = ctx.learn_train(1, batch=16, lr=1e-3, seed=1)
        last = ctx.learn_train(7, batch=16, lr=1e-3, seed=2)
        assert last < first
        ctx.learn_record(False)
        ctx.reset_to_seed()
        stats, rc = ctx.solve_all(1, 2)
        assert rc == 0 and len(stats) == 2 * wl.nrhs
        for st in stats:
            assert st["relres"] <= inp["tol"][st["rhs"]] * 1.0001, st
        assert sum(st["augmented"] for st in stats) > wl.nrhs
        for smp in (1, 2):
            A, Bt, Ct = op.assemble(inp, smp)
            B = np.hstack([Bt, Ct])
            Xs = ctx.solutions(smp)
            for j in (0, wl.nsrc - 1, wl.nsrc, wl.nrhs - 1):
                rr = np.linalg.norm(B[:, j] - A @ Xs[:, j]) / np.linalg.norm(B[:, j])
                assert rr <= inp["tol"][j] * 1.05, (smp, j, rr)
            del Xs, A
        plain = _ctx(rcg, inp, 2, precision=rcg.RCG_MIXED, order=rcg.RCG_WAVE, tau_rank=1e-6, r_max=1024)
        plain.seed_copy(ctx)
        stats_p, rc = plain.solve_all(1, 2)
        assert rc == 0
        it_l = np.mean([st["iters"] for st in stats])
        it_p = np.mean([st["iters"] for st in stats_p])
        print("mean CG iterations: learned", it_l, "plain", it_p)
        assert it_l < it_p, (it_l, it_p)
        for smp in (1, 2):
            P_l = ctx.rom_eval(inp["mu"][smp])[0]
            P_p = plain.rom_eval(inp["mu"][smp])[0]
            assert _rel(P_l, P_p) <= 1e-6, (smp, _rel(P_l, P_p))
    finally:
        ctx.close()
        if plain is not None:
            plain.close()


def test_192_cubed_waves_of_one_sample(rcg):
    inp = make_workload("c5_3d192", K=2, with_dmu=False)
    wl = inp["wl"]
    ctx = _ctx(rcg, inp, 2, precision=rcg.RCG_MIXED, order=rcg.RCG_WAVE, wave_samples=1, tau_rank=1e-6,
               r_max=2048)
    try:
        seed = ctx.seed(0, None)
        assert ctx.rank() == wl.k_u + wl.nrhs
        stats, rc = ctx.solve_all(1, 2)
        assert rc == 0 and len(stats) == 2 * wl.nrhs
        for s in stats:
            assert s["relres"] <= inp["tol"][s["rhs"]] * 1.0001, s
        psi64 = _fp64_psi(rcg, inp, ctx, [1, 2])
        for smp, P in psi64.items():
            Pm = ctx.rom_eval(inp["mu"][smp])[0]
            assert _rel(Pm, P) <= 1e-6, (smp, _rel(Pm, P))
    finally:
        ctx.close()
