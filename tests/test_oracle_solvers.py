"""Pins of the oracle's solvers: Krylov solutions against direct factorisations,
deflated CG against plain CG (empty deflation space) and eigenpairs against
eigen-residuals and the ordering of the spectrum."""
import numpy as np
import pytest

from oracle import eigen, operator as op, solvers
from synthetic.phantom import make_workload


@pytest.fixture(scope="module")
def sys2d():
    inp = make_workload("t2d_24")
    At, Bt, Ct = op.assemble(inp, 1)
    return inp, At, Bt, Ct


def test_direct_solvers_agree(sys2d):
    inp, At, Bt, Ct = sys2d
    B = np.hstack([Bt, Ct])
    X1 = solvers.dense_solve(At, B)
    X2 = solvers.direct_solve(At, B)
    X3 = solvers.banded_cholesky_solve(At, B, bw=inp["dims"][0])
    assert np.allclose(X1, X2, rtol=0, atol=1e-12 * np.abs(X1).max())
    assert np.allclose(X1, X3, rtol=0, atol=1e-12 * np.abs(X1).max())


def test_cg_matches_direct(sys2d):
    _, At, Bt, _ = sys2d
    b = Bt[:, 0]
    x, its, rel = solvers.cg(At, b, 1e-12)
    xd = solvers.dense_solve(At, b)
    assert rel <= 1e-12
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    assert its > 10


def test_deflated_cg_reduces_to_cg_and_deflation_helps(sys2d):
    inp, At, Bt, _ = sys2d
    b = Bt[:, 1]
    bn = np.linalg.norm(b)
    x0, it0, _ = solvers.cg(At, b, 1e-10)
    x1, it1, r1 = solvers.deflated_cg(At, b, None, 1e-10, bn)
    assert it0 == it1 and np.allclose(x0, x1, rtol=0, atol=1e-14 * np.abs(x0).max())
    w, U = eigen.smallest_eigenpairs(At, 8)
    x2, it2, r2 = solvers.deflated_cg(At, b, U, 1e-10, bn)
    xd = solvers.dense_solve(At, b)
    assert r2 <= 1e-10 and np.linalg.norm(x2 - xd) <= 1e-7 * np.linalg.norm(xd)
    assert it2 < it1       # deflating the smallest eigenvalues shortens CG
    # deflation with a non-orthonormal, badly scaled basis of the same span
    Wbad = U @ np.triu(np.ones((8, 8))) * 1e3
    x3, it3, r3 = solvers.deflated_cg(At, b, Wbad, 1e-10, bn)
    assert r3 <= 1e-10 and abs(it3 - it2) <= 2


def test_eigenpairs(sys2d):
    _, At, _, _ = sys2d
    w, U = eigen.smallest_eigenpairs(At, 10)
    A = At.toarray()
    full = np.linalg.eigvalsh(A)
    assert np.allclose(w, full[:10], rtol=1e-12)
    assert np.linalg.norm(A @ U - U * w) <= 1e-12 * full[-1]
    # the sparse path (ARPACK) finds the same invariant subspace
    w2, U2 = eigen.smallest_eigenpairs(At, 10, dense_limit=10)
    assert np.allclose(w2, w, rtol=1e-9)
    s = np.linalg.svd(U.T @ U2, compute_uv=False)
    assert s.min() > 1 - 1e-8
