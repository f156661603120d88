"""GPU tests of rcg_basis_compress: Algorithm 1 (truncated-SVD global basis,
Sec. 4.2.2) applied to the solutions Algorithm 2 delivered, against the
oracle's Algorithm 1 (numpy SVD) on the same kept solutions.

The library takes the singular values from the float64 Gram S^T S (parallel
Jacobi).  An eigenvalue error of ~eps ||S||^2 moves sigma_i by
~eps sigma_1^2 / sigma_i and the i-th singular vector by ~eps sigma_1^2 /
(sigma_i^2 - sigma_{i+1}^2); with tau = 1e-4 the kept vectors are determined to
~1e-8, so the subspace bound is 1e-6 (float64 basis) and 1e-5 (float32 basis,
re-orthonormalised in float32 by the append).  Decisions inside a guard band
around tau sigma_1 are skipped, as in the other parity tests.
"""
import numpy as np
import pytest

from oracle import alg1, operator as op, rom
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


def _sin_angle(A, B):
    QA, _ = np.linalg.qr(A)
    QB, _ = np.linalg.qr(B)
    return float(np.linalg.norm(QA - QB @ (QB.T @ QA), 2))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_compress_matches_oracle_algorithm1(rcg, precision):
    name = "t3d_32"
    inp = workload(name)
    wl = inp["wl"]
    prec = rcg.RCG_MIXED if precision == "mixed" else rcg.RCG_FP64
    order = rcg.RCG_WAVE if prec else rcg.RCG_SEQUENTIAL
    ctx, _, _, rc, _ = gpu_run(name, prec, order, 1e-6 if prec else 1e-12)
    try:
        assert rc == 0
        r_alg2 = ctx.rank()
        blocks = [ctx.solutions(s) for s in range(wl.K + 1)]     # seed sample 0 and samples 1..K are kept
        tau = 1e-4
        V_o, s_o = alg1.global_basis_svd(blocks, 0, tau)
        r_g, s_g = ctx.basis_compress(0, tau)
        assert len(s_g) == len(s_o) == (wl.K + 1) * wl.nrhs
        big = s_o >= 1e-6 * s_o[0]
        assert np.max(np.abs(s_g[big] - s_o[big])) <= 1e-9 * s_o[0]
        band = (s_o > tau * s_o[0] / 1.05) & (s_o < tau * s_o[0] * 1.05)
        if not band.any():
            assert r_g == V_o.shape[1]
        assert r_g < r_alg2 or r_alg2 <= V_o.shape[1]
        V_g = ctx.basis()
        k = min(r_g, V_o.shape[1])
        assert _sin_angle(V_g[:, :k], V_o[:, :k]) <= (1e-5 if prec else 1e-6)
        assert np.max(np.abs(V_g.T @ V_g - np.eye(r_g))) <= (5e-5 if prec else 1e-10)
        # the reduced model through the compressed basis
        _, As, Bt, Ct = oracle_seed_inputs(name)
        for s in (1, wl.K):
            Pg, _ = ctx.rom_eval(inp["mu"][s])
            Po, _ = rom.rom_eval(V_o, As[s], Bt, Ct, inp["h"])
            assert rel(Pg, Po) <= (1e-5 if prec else 1e-8), (s, rel(Pg, Po))
        # Algorithm 2 continues on the compressed basis: every solution meets its tolerance
        stats, rc2 = ctx.solve_all(1, wl.K)
        assert rc2 == 0
        B = np.hstack([Bt, Ct])
        for st in stats:
            i, j = st["sample"], st["rhs"]
            x = ctx.solutions(i)[:, j]
            assert np.linalg.norm(B[:, j] - As[i] @ x) <= inp["tol"][j] * 1.0000001 * np.linalg.norm(B[:, j])
        # the seed state is now the compressed basis
        ctx.reset_to_seed()
        assert ctx.rank() == r_g
    finally:
        ctx.close()


def test_compress_rank_cap_and_errors(rcg):
    name = "t3d_32"
    inp = workload(name)
    wl = inp["wl"]
    ctx, _, _, rc, _ = gpu_run(name, rcg.RCG_MIXED, rcg.RCG_WAVE, 1e-6)
    try:
        blocks = [ctx.solutions(s) for s in range(wl.K + 1)]
        r, s = ctx.basis_compress(7, 1e-10)
        assert r == 7
        V_o, _ = alg1.global_basis_svd(blocks, 7, 1e-10)
        assert _sin_angle(ctx.basis(), V_o) <= 1e-5
        # Eckart-Young on the device's basis: the residual of S in range(V) is the dropped sigma mass
        S = np.hstack(blocks)
        V = ctx.basis()
        err2 = np.linalg.norm(S - V @ (V.T @ S), "fro") ** 2
        assert err2 <= np.sum(s[7:] ** 2) * (1 + 1e-3) + 1e-10 * s[0] ** 2
        with pytest.raises(rcg.RcgError) as e:
            ctx.basis_compress(0, -1.0)
        assert e.value.code == rcg.RCG_ERR_INVALID
        with pytest.raises(rcg.RcgError):
            ctx.basis_compress(0, 2.0)          # no singular value above 2 sigma_1
        assert ctx.rank() == 7                  # unchanged by the refused call
    finally:
        ctx.close()
    # without kept solutions
    ctx2, _, _, _, _ = gpu_run(name, rcg.RCG_MIXED, rcg.RCG_WAVE, 1e-6, keep_solutions=0)
    try:
        with pytest.raises(rcg.RcgError) as e:
            ctx2.basis_compress(0, 1e-6)
        assert e.value.code == rcg.RCG_ERR_INVALID
    finally:
        ctx2.close()
