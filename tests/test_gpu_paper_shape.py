"""The paper's experiment shape on the GPU: 2D 201^2 (40401 unknowns), 32
sources + 32 detectors, three systems, tolerance 1e-7, float64, the paper's
order, its minimum-residual check and recycled MINRES (Sec. 6; Algorithm 2),
against per-RHS recycling only (the comparison method of Table 2).

The phantoms are synthetic stand-ins (the paper's are not published), so the
iteration counts differ from Tables 1 and 2; what is checked is the pattern
the paper reports and explains:
  * inner-outer recycling: within each half of the right-hand sides of a
    system (sources, then detectors) the MINRES iterations fall, to at most a
    fifth of the half's first count at its last right-hand side (Table 1: 140,
    52, 0).  The paper's jump at the first detector (RHS 33) does not occur
    here: the parameter points are small jitters of the seed point, and the
    directions the source half appends also serve the adjoint half (measured:
    61 MINRES iterations at RHS 1 of the first system, 3 at RHS 33), so the
    test does not require it;
  * per-RHS recycling does not speed up along the right-hand sides (Table 2's
    right columns: the last eight of a half need at least half the iterations
    of its first eight), while the inner-outer method does (its last eight
    need fewer than its first eight, and a smaller share of them than the
    per-RHS method's), and per-RHS recycling needs more than twice the total
    iterations (5006 against 22659 in the paper);
  * every delivered solution meets its tolerance under the oracle's residual;
  * the basis holds k_u + the seed solutions + one column per appended solve.
"""
import numpy as np
import pytest

from oracle import operator as op
from synthetic.phantom import make_workload

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


def _run(rcg, inp, recycle):
    wl = inp["wl"]
    ctx = rcg.Context(wl.dim, wl.N, wl.robin_A, precision=rcg.RCG_FP64, order=rcg.RCG_SEQUENTIAL, tau_rank=1e-12,
                      k_u=wl.k_u, keep_solutions=1, check=rcg.RCG_MR, inner=rcg.RCG_MINRES, recycle=recycle)
    ctx.set_diffusion(inp["D"])
    ctx.set_sources_detectors(inp["src_ij"], inp["det_ij"])
    ctx.set_tolerances(inp["tol"])
    for s in range(wl.K + 1):
        ctx.set_sample(s, inp["mu"][s])
    ctx.seed(0, None)
    stats, rc = ctx.solve_all(1, wl.K)
    return ctx, stats, rc


def test_paper_shape_table1_pattern_and_table2_direction(rcg):
    inp = make_workload("paper_2d201")
    wl = inp["wl"]
    m, ns = wl.nrhs, wl.nsrc
    ctx, io, rc = _run(rcg, inp, rcg.RCG_INNER_OUTER)
    try:
        assert rc == 0
        for s in range(1, wl.K + 1):
            A, Bt, Ct = op.assemble(inp, s)
            B = np.hstack([Bt, Ct])
            X = ctx.solutions(s)
            rr = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
            assert np.all(rr <= inp["tol"] * 1.05), (s, rr.max())
        assert ctx.rank() == wl.k_u + m + sum(o["appended"] for o in io)
    finally:
        ctx.close()
    ctx2, pr, rc2 = _run(rcg, inp, rcg.RCG_PER_RHS)
    try:
        assert rc2 == 0
        X = ctx2.solutions(wl.K)
        A, Bt, Ct = op.assemble(inp, wl.K)
        B = np.hstack([Bt, Ct])
        rr = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
        assert np.all(rr <= inp["tol"] * 1.05), rr.max()
    finally:
        ctx2.close()
    it_io = [o["iters"] for o in io]
    it_pr = [o["iters"] for o in pr]
    for i in range(wl.K):
        seg = it_io[i * m:(i + 1) * m]
        assert seg[ns - 1] <= 0.2 * seg[0] and seg[-1] <= 0.2 * max(seg[ns], 1), seg
        assert seg[19] < seg[0] if i == 0 else seg[19] <= seg[0], seg    # RHS 20 of Table 1
        # per-RHS recycling does not speed up along the right-hand sides of a half
        pseg = it_pr[i * m:(i + 1) * m]
        for h0 in (0, ns):
            first, last = np.mean(pseg[h0:h0 + 8]), np.mean(pseg[h0 + ns - 8:h0 + ns])
            assert last >= 0.5 * first, (i, h0, pseg)
            # inner-outer: the half speeds up, by more than per-RHS recycling does
            io_first, io_last = np.mean(seg[h0:h0 + 8]), np.mean(seg[h0 + ns - 8:h0 + ns])
            assert io_last < io_first, (i, h0, seg)
            assert io_last / io_first < last / first, (i, h0, seg, pseg)
    assert 2 * sum(it_io) < sum(it_pr), (sum(it_io), sum(it_pr), it_io, it_pr)
