"""Smallest eigenpairs of A~_0 for the seed recycle space U_0 (Sec. 4.2.2,
Algorithm 2 first step: 10 eigenvectors of A~_0 for the smallest eigenvalues).

The paper does not name its eigensolver (it speaks of estimates).  The oracle
uses LAPACK's dense symmetric solver (numpy.linalg.eigh) on small grids and
ARPACK's implicitly restarted Lanczos (scipy eigsh) otherwise.
Parity: pinned by the constant-coefficient closed-form spectrum (a Kronecker
sum of 1-D tridiagonals) and by eigen-residual checks.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def smallest_eigenpairs(A, k, dense_limit=4096, tol=1e-12, seed=0):
    n = A.shape[0]
    if n <= dense_limit:
        w, U = np.linalg.eigh(A.toarray() if sp.issparse(A) else np.asarray(A))
        return w[:k], U[:, :k]
    v0 = np.random.default_rng(seed).standard_normal(n)
    w, U = spla.eigsh(sp.csr_matrix(A), k=k, which="SA", tol=tol, v0=v0,
                      ncv=max(4 * k, 40), maxiter=200000)
    order = np.argsort(w)
    return w[order], U[:, order]
