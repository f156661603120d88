"""Parity at the bench workload's full size (3D 64^3, 32 + 32 right-hand
sides, 5 samples) in the bench's launch configuration: learned + mixed wave,
device eigen seed, the network trained on held-out parameter points.

The oracle cannot replay 320 solves at this size in seconds, so it checks
what holds at any size, on samples of the outputs:
* sampled delivered solutions: residual recomputed by the oracle's operator
  (scipy, float64) within the right-hand side's tolerance;
* the basis is orthonormal to float32 accuracy;
* the reduced model at a sampled parameter point equals the oracle's reduced
  model built from the same basis, and interpolates the full-order transfer
  function of the delivered solutions (Sec. 3.4).
"""
import numpy as np
import pytest

from oracle import operator as op, rom
from synthetic.cnn_init import init_weights
from synthetic.phantom import heldout_params, make_workload, pals_mu, pals_dmu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1602_00138_gb300 import rcg
    inp = make_workload("c2_3d64")
    wl = inp["wl"]
    K = wl.K
    ntr = 2
    ctx = rcg.Context(wl.dim, wl.N, wl.robin_A, k_u=wl.k_u, max_samples=K + 1 + ntr, r_max=1024,
                      precision=rcg.RCG_MIXED, order=rcg.RCG_WAVE, tau_rank=1e-6, learned=1, keep_solutions=1)
    ctx.set_diffusion(inp["D"])
    ctx.set_sources_detectors(inp["src_ij"], inp["det_ij"])
    ctx.set_tolerances(inp["tol"])
    for s in range(K + 1):
        ctx.set_sample(s, inp["mu"][s])
    for i, p in enumerate(heldout_params(wl, ntr, seed_offset=2000)):
        ctx.set_sample(K + 1 + i, pals_mu(p, inp["X"], wl.mu_bg))
    ctx.seed(0, None)
    ctx.learn_set_weights(init_weights(0))
    ctx.learn_record(True)
    ctx.solve_all(K + 1, ntr)
    ctx.learn_train(10, 16, 1e-3, 1)
    ctx.learn_record(False)
    ctx.reset_to_seed()
    stats, rc = ctx.solve_all(1, K)
    yield rcg, inp, ctx, stats, rc
    ctx.close()


def test_sampled_solutions_meet_tolerance(run):
    rcg, inp, ctx, stats, rc = run
    wl = inp["wl"]
    assert rc == 0 and len(stats) == wl.K * wl.nrhs
    assert sum(s["augmented"] for s in stats) > 0
    rng = np.random.default_rng(5)
    picks = {(1, 0), (wl.K, wl.nrhs - 1)} | {(int(rng.integers(1, wl.K + 1)), int(rng.integers(0, wl.nrhs)))
                                             for _ in range(8)}
    for i in sorted({i for i, _ in picks}):
        At, Bt, Ct = op.assemble(inp, i)
        B = np.hstack([Bt, Ct])
        X = ctx.solutions(i)
        for (ii, j) in picks:
            if ii != i:
                continue
            res = np.linalg.norm(B[:, j] - At @ X[:, j]) / np.linalg.norm(B[:, j])
            assert res <= inp["tol"][j] * 1.0000001, (i, j, res)


def test_basis_is_orthonormal(run):
    rcg, inp, ctx, stats, rc = run
    V = ctx.basis()
    G = V.T @ V
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 5e-5


def test_reduced_model_matches_oracle_and_interpolates(run):
    rcg, inp, ctx, stats, rc = run
    wl = inp["wl"]
    i = 3
    At, Bt, Ct = op.assemble(inp, i)
    V = ctx.basis()
    dmu = np.asarray(pals_dmu(inp["params"][i], inp["X"], wl.mu_bg))
    Psi, J = ctx.rom_eval(inp["mu"][i], dmu)
    Psi_o, J_o = rom.rom_eval(V, At, Bt, Ct, wl.h, dmu)
    assert np.linalg.norm(Psi - Psi_o) <= 1e-6 * np.linalg.norm(Psi_o)
    assert np.linalg.norm(J - J_o) <= 1e-6 * np.linalg.norm(J_o)     # the same basis: the mixed acceptance tolerance
    # interpolation at a sampled point: C~^T x of the delivered source solutions.
    # Those carry their own error (relres <= 1e-8, amplified by A~^-1 up to
    # ~kappa), so the bound is 1e-5 relative; a basis without the sampled
    # solutions misses by orders of magnitude more.
    Xall = ctx.solutions(i)
    X, Z = Xall[:, :wl.nsrc], Xall[:, wl.nsrc:]
    Psi_full, J_full = ctx.full_eval(i, dmu)
    # rcg_full_eval is the plain definition on the delivered solutions (Sec. 3.1, eq. newjac)
    assert np.allclose(Psi_full, Ct.T @ X, rtol=1e-12, atol=0)
    J_ref = np.stack([-(Z.T @ ((wl.h * wl.h * dmu[k])[:, None] * X)) for k in range(dmu.shape[0])])
    assert np.linalg.norm(J_full - J_ref) <= 1e-10 * np.linalg.norm(J_ref)
    err = np.linalg.norm(Psi - Psi_full) / np.linalg.norm(Psi_full)
    assert err <= 1e-5, err
    errJ = np.linalg.norm(J - J_full) / np.linalg.norm(J_full)
    assert errJ <= 1e-3, errJ
