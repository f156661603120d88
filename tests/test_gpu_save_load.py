"""GPU tests of rcg_save / rcg_load (the recycling state carried to another
context) and rcg_full_eval on a small workload.

A context that loads the saved state must hold the same basis, reduced model
and seed state as the one that saved it, continue Algorithm 2 from it with
every solution within tolerance, and refuse a state saved for different
inputs.
"""
import os

import numpy as np
import pytest

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


def _ctx(rcg, inp, D=None):
    wl = inp["wl"]
    ctx = rcg.Context(wl.dim, wl.N, wl.robin_A, precision=rcg.RCG_MIXED, order=rcg.RCG_WAVE, k_u=wl.k_u,
                      tau_rank=1e-6, keep_solutions=1)
    ctx.set_diffusion(inp["D"] if D is None else D)
    ctx.set_sources_detectors(inp["src_ij"], inp["det_ij"])
    ctx.set_tolerances(inp["tol"])
    return ctx


def test_saved_state_reloads_and_continues(rcg, tmp_path):
    inp = workload("t3d_32")
    wl = inp["wl"]
    U0, As, Bt, Ct = oracle_seed_inputs("t3d_32")
    a = _ctx(rcg, inp)
    b = _ctx(rcg, inp)
    try:
        for s in range(wl.K + 1):
            a.set_sample(s, inp["mu"][s])
        a.seed(0, U0)
        a.learn_set_weights(init_weights(3))
        r_seed = a.rank()
        a.solve_all(1, wl.K)
        path = os.path.join(str(tmp_path), "state.rcg")
        a.save(path)
        for s in range(1, wl.K + 1):
            b.set_sample(s, inp["mu"][s])
        b.load(path)
        assert b.rank() == a.rank()
        assert np.array_equal(b.basis(), a.basis())
        assert np.array_equal(b.learn_get_weights(), init_weights(3))
        Pa, _ = a.rom_eval(inp["mu"][2])
        Pb, _ = b.rom_eval(inp["mu"][2])
        assert np.allclose(Pa, Pb, rtol=1e-12, atol=0)
        # continue Algorithm 2 on the loaded state (samples already represented: V suffices mostly)
        stats, rc = b.solve_all(1, wl.K)
        assert rc == 0
        B = np.hstack([Bt, Ct])
        for st in stats:
            i, j = st["sample"], st["rhs"]
            x = b.solutions(i)[:, j]
            assert np.linalg.norm(B[:, j] - As[i] @ x) <= inp["tol"][j] * 1.0000001 * np.linalg.norm(B[:, j])
        b.reset_to_seed()
        assert b.rank() == r_seed
        # full-order transfer function of the delivered solutions
        Psi, _ = b.full_eval(2)
        X = b.solutions(2)
        assert np.allclose(Psi, Ct.T @ X[:, :wl.nsrc], rtol=1e-12, atol=0)
    finally:
        a.close()
        b.close()


def test_state_of_other_inputs_is_refused(rcg, tmp_path):
    inp = workload("t3d_32")
    wl = inp["wl"]
    U0 = oracle_seed_inputs("t3d_32")[0]
    a = _ctx(rcg, inp)
    b = _ctx(rcg, inp, D=inp["D"] * 1.01)
    try:
        a.set_sample(0, inp["mu"][0])
        a.seed(0, U0)
        path = os.path.join(str(tmp_path), "state.rcg")
        a.save(path)
        with pytest.raises(rcg.RcgError) as e:
            b.load(path)
        assert e.value.code == rcg.RCG_ERR_INVALID
        with pytest.raises(rcg.RcgError):
            b.load(os.path.join(str(tmp_path), "missing.rcg"))
    finally:
        a.close()
        b.close()
