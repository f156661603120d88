"""GPU tests of rcg_rom_eval_batch: the reduced transfer function Psi_r and
its Jacobian (eq. newreduced, eq. newjac) at many parameter points in one
call, the evaluation the optimisation of Sec. 4.2.2 repeats through a fixed V.

References: the oracle's reduced model built from the context's own basis
(a float64 Galerkin projection with dense Cholesky), and rcg_rom_eval at
each point.  Mixed precision forms the weighted Grams on the tensor cores
(3xTF32 products, float64 slice sums); on the context's own basis the bounds
are the acceptance tolerances: 1e-6 relative for Psi_r and J (mixed),
1e-10 / 1e-9 (float64).  Held-out points
(not used to build V) and the sampled points are both covered; a point
count that is not a multiple of anything and nq = 0 are edge cases.
"""
import numpy as np
import pytest

from oracle import operator as op, rom
from synthetic.phantom import heldout_params, pals_dmu, pals_mu
from tests.gpu_common import gpu_run, oracle_seed_inputs, workload

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _points(name, count):
    inp = workload(name)
    wl = inp["wl"]
    ps = list(heldout_params(wl, count))
    ps.append(inp["params"][2])                      # one sampled point as well
    mus = np.stack([pals_mu(p, inp["X"], wl.mu_bg) for p in ps])
    dmus = np.stack([pals_dmu(p, inp["X"], wl.mu_bg) for p in ps])
    return inp, mus, dmus


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_matches_single_points_and_oracle(rcg, precision):
    name = "t3d_32"
    inp, mus, dmus = _points(name, 6)
    wl = inp["wl"]
    prec = rcg.RCG_MIXED if precision == "mixed" else rcg.RCG_FP64
    ctx, _, _, rc, _ = gpu_run(name, prec, rcg.RCG_WAVE, 1e-6 if prec else 1e-12)
    try:
        assert rc == 0
        V = ctx.basis()
        _, _, Bt, Ct = oracle_seed_inputs(name)
        Psi_b, J_b = ctx.rom_eval_batch(mus, dmus)
        assert Psi_b.shape == (len(mus), wl.ndet, wl.nsrc)
        assert J_b.shape == (len(mus), dmus.shape[1], wl.ndet, wl.nsrc)
        psi_tol, j_tol = (1e-6, 1e-6) if prec else (1e-10, 1e-9)
        for q in range(len(mus)):
            Pq, Jq = ctx.rom_eval(mus[q], dmus[q])
            A = op.schur_for_mu(inp, mus[q])
            Po, Jo = rom.rom_eval(V, A, Bt, Ct, inp["h"], dmus[q])
            assert rel(Psi_b[q], Po) <= psi_tol, (q, rel(Psi_b[q], Po))
            assert rel(J_b[q], Jo) <= j_tol, (q, rel(J_b[q], Jo))
            assert rel(Psi_b[q], Pq) <= psi_tol and rel(J_b[q], Jq) <= j_tol
            if not prec:        # the float64 path evaluates the points one by one through rcg_rom_eval
                # (its Jacobian products sum split-K slices with float64 atomics: equal up to ordering)
                assert rel(Psi_b[q], Pq) <= 1e-12 and rel(J_b[q], Jq) <= 1e-12
        # without the Jacobian
        Psi_n, J_n = ctx.rom_eval_batch(mus[:3])
        assert J_n is None and np.allclose(Psi_n, Psi_b[:3], rtol=1e-12, atol=0)
    finally:
        ctx.close()


def test_batch_edge_cases(rcg):
    import torch
    name = "t3d_32"
    inp, mus, dmus = _points(name, 2)
    ctx, _, _, rc, _ = gpu_run(name, rcg.RCG_MIXED, rcg.RCG_WAVE, 1e-6)
    try:
        # nq = 0: nothing to do
        z = torch.zeros(1, dtype=torch.float64, device="cuda")
        assert ctx.rom_eval_batch_device(0, z, None, z, None, 0) == 0
        # J requested without dmu, negative nq: refused
        with pytest.raises(rcg.RcgError) as e:
            ctx.rom_eval_batch_device(1, torch.from_numpy(mus[:1]).cuda(), None, torch.zeros(64, dtype=torch.float64,
                                      device="cuda"), z, 3)
        assert e.value.code == rcg.RCG_ERR_INVALID
        with pytest.raises(rcg.RcgError):
            ctx.rom_eval_batch_device(-1, z, None, z, None, 0)
        # a single point equals rcg_rom_eval
        P1, J1 = ctx.rom_eval_batch(mus[:1], dmus[:1])
        Pq, Jq = ctx.rom_eval(mus[0], dmus[0])
        assert rel(P1[0], Pq) <= 1e-6 and rel(J1[0], Jq) <= 1e-6
    finally:
        ctx.close()


def test_batch_of_more_points_than_one_chunk(rcg):
    """257 points: more than one chunk of rcg_rom_eval_batch (at most 256
    points per chunk), so the second chunk's offsets into mu, dmu, Psi and J
    are exercised; every point equals rcg_rom_eval at that point."""
    name = "t3d_32"
    inp = workload(name)
    wl = inp["wl"]
    ps = heldout_params(wl, 257, seed_offset=3000)
    mus = np.stack([pals_mu(p, inp["X"], wl.mu_bg) for p in ps])
    dmus = np.stack([pals_dmu(p, inp["X"], wl.mu_bg) for p in ps])
    ctx, _, _, rc, _ = gpu_run(name, rcg.RCG_MIXED, rcg.RCG_WAVE, 1e-6)
    try:
        assert rc == 0
        Psi_b, J_b = ctx.rom_eval_batch(mus, dmus)
        for q in (0, 1, 128, 255, 256):
            Pq, Jq = ctx.rom_eval(mus[q], dmus[q])
            assert rel(Psi_b[q], Pq) <= 1e-6 and rel(J_b[q], Jq) <= 1e-6, q
        # the chunks do not bleed: the last point differs from its neighbour where their parameters do
        assert rel(Psi_b[256], Psi_b[255]) > 1e-9
    finally:
        ctx.close()
