"""Pins of the oracle's minimum-residual check and recycled MINRES
(oracle/minres.py; Sec. 4.1 eqs. initialz, eq01, SmallMin; Algorithm 2) and
of the per-RHS recycling comparison of Sec. 6.3 (Table 2), against facts
independent of the recurrences: dense least-squares minimisers over the
defining subspaces, direct solves, and the iteration pattern of Table 2."""
import numpy as np
import pytest

from oracle import basis, eigen, minres, operator as op, solvers
from synthetic.phantom import make_workload


@pytest.fixture(scope="module")
def system():
    inp = make_workload("t2d_24")
    A, Bt, Ct = op.assemble(inp, 1)
    return inp, A, Bt, Ct


def test_mr_check_is_the_least_squares_minimiser(system):
    """z = U K^T b minimises ||b - A x|| over range(V) (eq. initialz): the
    same point as a dense least-squares solve with the columns A V."""
    inp, A, Bt, Ct = system
    rng = np.random.default_rng(2)
    V, _ = np.linalg.qr(rng.standard_normal((A.shape[0], 9)))
    b = Ct[:, 1]
    z, r, rel = minres.mr_check(A, V, b)
    y, *_ = np.linalg.lstsq((A @ V), b, rcond=None)
    assert np.linalg.norm(z - V @ y) <= 1e-10 * np.linalg.norm(z)
    assert np.allclose(r, b - A @ z, rtol=0, atol=1e-14 * np.linalg.norm(b))
    assert np.isclose(rel, np.linalg.norm(b - A @ (V @ y)) / np.linalg.norm(b), rtol=1e-9)


def _reference_iterate(A, r, U, m):
    """argmin ||r - A g|| over range([U, K_m]) with K_m the Krylov space of
    P A P from P r (P the orthogonal projector away from range(A U)), built
    by Arnoldi with full reorthogonalisation and solved by dense least
    squares: the definition of the m-th recycled MINRES iterate."""
    n = A.shape[0]
    Ad = A.toarray()
    if U.shape[1]:
        K, _ = np.linalg.qr(Ad @ U)
        P = np.eye(n) - K @ K.T
    else:
        P = np.eye(n)
    Q = [P @ r / np.linalg.norm(P @ r)]
    for _ in range(m - 1):
        w = P @ (Ad @ Q[-1])
        for _rep in range(2):
            for q in Q:
                w = w - (q @ w) * q
        Q.append(w / np.linalg.norm(w))
    S = np.column_stack([U] + [q[:, None] for q in Q]) if U.shape[1] else np.column_stack(Q)
    c, *_ = np.linalg.lstsq(Ad @ S, r, rcond=None)
    return S @ c


@pytest.mark.parametrize("k", [0, 4])
def test_every_minres_iterate_minimises_the_residual_over_its_space(system, k):
    inp, A, Bt, Ct = system
    rng = np.random.default_rng(3)
    _, U0 = eigen.smallest_eigenpairs(A, 6)
    U = U0[:, :k] + 1e-3 * rng.standard_normal((A.shape[0], k))     # a recycle space near an invariant one
    r = Bt[:, 2] + 0.1 * rng.standard_normal(A.shape[0])
    Uh, K = minres.recycle_basis(A, U)
    trace = []
    g, its, phibar = minres.minres_cycle(A, r, Uh, K, 0.0, 12, trace)
    assert its == 12 and len(trace) == 12
    for m in (1, 2, 5, 12):
        ref = _reference_iterate(A, r, U, m)
        assert np.linalg.norm(trace[m - 1] - ref) <= 1e-8 * np.linalg.norm(ref), m
    # |phibar| is the true residual norm of the iterate
    assert np.isclose(phibar, np.linalg.norm(r - A @ g), rtol=1e-8)


def test_recycled_minres_reaches_the_direct_solution(system):
    inp, A, Bt, Ct = system
    b = Bt[:, 0]
    bn = np.linalg.norm(b)
    xd = solvers.direct_solve(A, b)
    g0, its0, rel0 = minres.recycled_minres(A, b, np.zeros((A.shape[0], 0)), 1e-11, bn)
    _, U0 = eigen.smallest_eigenpairs(A, 6)
    g1, its1, rel1 = minres.recycled_minres(A, b, U0, 1e-11, bn)
    for g, rel in ((g0, rel0), (g1, rel1)):
        assert rel <= 1e-11 and np.linalg.norm(b - A @ g) / bn <= 1e-11
        assert np.linalg.norm(g - xd) <= 1e-8 * np.linalg.norm(xd)
    assert its1 < its0                              # the smallest eigenvectors deflated: fewer iterations


def test_table2_direction_inner_outer_against_per_rhs_recycling():
    """Sec. 6.3 / Table 2: with the paper's own check and inner solver, the
    inner-outer method's iterations fall along the right-hand sides of each
    half (sources, detectors) and reach few or none at the end of a half,
    with a jump at the first detector; per-RHS recycling alone keeps roughly
    the same count for every right-hand side and needs several times more
    iterations in total."""
    inp = make_workload("t2d_48")           # 2D 48^2, 12 sources + 12 detectors, 2 samples
    wl = inp["wl"]
    A0, Bt, Ct = op.assemble(inp, 0)
    B = np.hstack([Bt, Ct])
    tols = inp["tol"]
    _, U0 = eigen.smallest_eigenpairs(A0, wl.k_u)
    As = {i: op.assemble(inp, i)[0] for i in range(1, wl.K + 1)}
    st = basis.seed(A0, B, U0, tols, inner="minres")
    io = basis.solve_all(st, lambda i: As[i], range(1, wl.K + 1), B, tols, check="mr", inner="minres")
    st2 = basis.seed(A0, B, U0, tols, inner="minres")
    pr = basis.solve_all_per_rhs(st2, lambda i: As[i], range(1, wl.K + 1), B, tols)
    for o in io + pr:
        b = B[:, o["rhs"]]
        assert o["relres"] <= tols[o["rhs"]] * 1.0000001
    it_io = [o["iters"] for o in io]
    it_pr = [o["iters"] for o in pr]
    assert sum(it_io) * 2 < sum(it_pr)
    m, ns = B.shape[1], wl.nsrc
    for i in range(wl.K):
        seg = it_io[i * m:(i + 1) * m]
        assert seg[ns - 1] < 0.5 * seg[0] and seg[-1] < 0.5 * seg[ns]     # falls within each half
        assert seg[ns] > seg[ns - 1]                                        # jump at the first detector
        pseg = it_pr[i * m:(i + 1) * m]
        assert min(pseg) > 0.5 * max(pseg)                                  # no such decrease
    # rank: k_u + every seed solution + one column per inner-outer solve that appended
    assert st.r == wl.k_u + wl.nrhs + sum(o["appended"] for o in io)
