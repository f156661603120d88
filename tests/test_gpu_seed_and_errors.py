"""GPU tests of the on-device eigen seed and of the library's error paths.

Eigen seed (Sec. 4.2.2: U_0 = eigenvectors of A~_0 for its smallest
eigenvalues): the first k_u columns of V after rcg_seed(U0 = NULL) must span
the oracle's invariant subspace (principal angles ~ 0) and satisfy the
eigen-residual bound.  Error paths: failures are produced on the host (bad
arguments, an iteration cap, a basis cap); no device fault is involved.
"""
import numpy as np
import pytest

from oracle import eigen, operator as op
from tests.gpu_common import workload

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


def _ctx(rcg, name, **opts):
    inp = workload(name)
    wl = inp["wl"]
    ctx = rcg.Context(wl.dim, wl.N, wl.robin_A, k_u=wl.k_u, **opts)
    ctx.set_diffusion(inp["D"])
    ctx.set_sources_detectors(inp["src_ij"], inp["det_ij"])
    ctx.set_tolerances(inp["tol"])
    for s in range(wl.K + 1):
        ctx.set_sample(s, inp["mu"][s])
    return inp, ctx


@pytest.mark.parametrize("name,prec", [("t3d_21", 0), ("t3d_32", 1), ("t2d_37", 0)])
def test_device_eigen_seed_spans_smallest_eigenvectors(rcg, name, prec):
    inp, ctx = _ctx(rcg, name, precision=prec)
    wl = inp["wl"]
    try:
        stats = ctx.seed(0, None)
        assert ctx.rank() == wl.k_u + wl.nrhs
        assert all(s["relres"] <= inp["tol"][s["rhs"]] * 1.0000001 for s in stats)
        V = ctx.basis()
        U = V[:, :wl.k_u]
        A0, _, _ = op.assemble(inp, 0)
        w, Uo = eigen.smallest_eigenpairs(A0, wl.k_u)
        # principal angles between the two k_u-dimensional subspaces
        sv = np.linalg.svd(U.T @ Uo, compute_uv=False)
        tol_angle = 1e-6 if prec == 0 else 1e-3
        assert sv.min() > 1 - tol_angle, sv
        # Rayleigh-Ritz residual of the device subspace
        H = U.T @ (A0 @ U)
        th, Y = np.linalg.eigh(H)
        Ur = U @ Y
        res = np.linalg.norm(A0 @ Ur - Ur * th, axis=0).max()
        lmax = abs(A0).sum(axis=1).max()
        assert res <= (1e-8 if prec == 0 else 1e-4) * lmax, res
        assert np.allclose(th, w, rtol=1e-6 if prec == 0 else 1e-3)
    finally:
        ctx.close()


def test_invalid_arguments_are_rejected(rcg):
    inp = workload("t2d_24")
    wl = inp["wl"]
    with rcg.Context(wl.dim, wl.N, wl.robin_A, k_u=wl.k_u) as ctx:
        with pytest.raises(rcg.RcgError) as e:
            ctx.set_sources_detectors(inp["src_ij"], inp["det_ij"])     # before D
        assert e.value.code == rcg.RCG_ERR_INVALID
        bad = inp["D"].copy()
        bad[5] = -1.0
        with pytest.raises(rcg.RcgError):
            ctx.set_diffusion(bad)                                      # D must be > 0
        ctx.set_diffusion(inp["D"])
        mu = inp["mu"][0].copy()
        mu[3] = np.nan
        with pytest.raises(rcg.RcgError):
            ctx.set_sample(0, mu)                                       # mu must be finite
        ctx.set_sources_detectors(inp["src_ij"], inp["det_ij"])
        with pytest.raises(rcg.RcgError):
            ctx.set_tolerances(np.full(wl.nrhs, 2.0))                   # tol in (0, 1)
        with pytest.raises(rcg.RcgError):
            ctx.solve_all(1, 1)                                         # sample not set / no seed
        bad_ij = np.array(inp["src_ij"]).copy()
        bad_ij[0, 0] = wl.N + 5
        with pytest.raises(rcg.RcgError):
            ctx.set_sources_detectors(bad_ij, inp["det_ij"])            # face point out of range


def test_iteration_cap_reports_not_converged_with_stats(rcg):
    inp, ctx = _ctx(rcg, "t2d_24", maxit=3)
    wl = inp["wl"]
    try:
        U0 = eigen.smallest_eigenpairs(op.assemble(inp, 0)[0], wl.k_u)[1]
        ctx.seed(0, U0)
        stats, rc = ctx.solve_all(1, 1)
        assert rc == rcg.RCG_ERR_NOT_CONVERGED
        capped = [s for s in stats if s["status"] == rcg.RCG_ERR_NOT_CONVERGED]
        assert capped and all(s["iters"] >= 3 for s in capped)
        assert all(np.isfinite(s["relres"]) for s in stats)
    finally:
        ctx.close()


def test_rank_cap_is_reported(rcg):
    inp, ctx = _ctx(rcg, "t2d_24", r_max=12)
    wl = inp["wl"]
    try:
        U0 = eigen.smallest_eigenpairs(op.assemble(inp, 0)[0], wl.k_u)[1]
        with pytest.raises(rcg.RcgError) as e:
            ctx.seed(0, U0)                                              # 6 + 8 columns > 12
        assert e.value.code == rcg.RCG_ERR_RANK_CAP
    finally:
        ctx.close()


def test_tiny_spin_budget_times_out_and_the_gpu_stays_usable(rcg):
    """rcg_options.spin_budget bounds the tensor-core kernels' main-loop
    waits for their MMAs.  A negative budget allows no poll, so the first such
    wait runs out (a step's MMAs usually complete within one poll, which would
    not exercise the path); the kernel then stops issuing, waits with its full
    bound for the last MMAs it committed, frees its tensor memory and reports
    RCG_ERR_TIMEOUT, which the call returns.  A context created afterwards with
    the default budget runs the same seed normally."""
    inp, ctx = _ctx(rcg, "t3d_32", precision=rcg.RCG_MIXED, order=rcg.RCG_WAVE, tau_rank=1e-6, spin_budget=-1)
    try:
        with pytest.raises(rcg.RcgError) as e:
            ctx.seed(0, None)
        assert e.value.code == rcg.RCG_ERR_TIMEOUT
    finally:
        ctx.close()
    inp, ctx = _ctx(rcg, "t3d_32", precision=rcg.RCG_MIXED, order=rcg.RCG_WAVE, tau_rank=1e-6)
    try:
        ctx.seed(0, None)
        stats, rc = ctx.solve_all(1, 1)
        assert rc == 0
        for st in stats:                                   # tolerances alternate 1e-8 / 1e-6 over the RHS
            assert st["relres"] <= inp["tol"][st["rhs"]] * 1.0001, st
    finally:
        ctx.close()
