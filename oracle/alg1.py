"""Algorithm 1 of the paper ("Generate Symmetric Global Basis via Truncated
SVD", Sec. 4.2.2) restated in float64.  Test infrastructure: only the tests,
the smoke check and the bench's CPU legs use this module.

    1. solve A~(p_k) X_k = [B~, C~] for the K parameter vectors p_1 .. p_K;
    2. concatenate the block solutions, S = [X_1, X_2, ..., X_K];
    3. V = the first r left singular vectors of S.

The paper leaves r to the user.  This restatement (and the library's
rcg_basis_compress, which applies steps 2-3 to the delivered solutions of
Algorithm 2) takes r = min(r_max, #{i : sigma_i > tau sigma_1}): the
numerical rank of S at relative level tau, capped.

Step 1 here is a direct solve per sample (the plain definition of X_k); the
library uses the solutions its recycled solves delivered, which meet the
same systems to their tolerance.

Pins (tests/test_oracle_alg1.py): snapshot matrices with prescribed singular
values (the rank rule and the subspace follow from the SVD by construction),
the Eckart-Young error ||S - V V^T S||_F^2 = sum_{i>r} sigma_i^2, invariance
under repeated columns, and the interpolation property of V when r is the full
rank (Psi_r = Psi at every sampled point).
"""
from __future__ import annotations

import numpy as np

from .solvers import direct_solve


def snapshot_solves(As, B):
    """Step 1: X_k = A~_k^-1 B for every matrix in As (dense or sparse)."""
    return [direct_solve(A, B) for A in As]


def truncation_rank(sigma, r_max, tau):
    """r = min(r_max, #{sigma_i > tau sigma_1}); r_max <= 0 means no cap."""
    sigma = np.asarray(sigma, dtype=np.float64)
    if sigma.size == 0 or sigma[0] <= 0.0:
        return 0
    r = int(np.count_nonzero(sigma > tau * sigma[0]))
    return min(r, r_max) if r_max > 0 else r


def global_basis_svd(blocks, r_max, tau):
    """Steps 2-3: V (n x r) and the singular values of S = [X_1, ..., X_K]."""
    S = np.hstack([np.asarray(X, dtype=np.float64) for X in blocks])
    U, sigma, _ = np.linalg.svd(S, full_matrices=False)
    r = truncation_rank(sigma, r_max, tau)
    return U[:, :r], sigma
