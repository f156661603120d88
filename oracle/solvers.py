"""Direct and Krylov solvers for the SPD Schur system A~ x = b (float64).

* `direct_solve`: sparse LU (SuperLU) of A~ -- the plain definition
  x = A~^-1 b used for exact targets (Sec. 3.3 eq. solves, Sec. 3.4 Theorem).
* `dense_solve`: numpy dense solve, for tiny grids.
* `banded_cholesky_solve`: Cholesky of the band of A~ in natural ordering
  (2D grids; the band width is Nx).
* `cg`: plain conjugate gradients (Hestenes-Stiefel).
* `deflated_cg`: deflated CG of Saad, Yeung, Erhel & Guyomarc'h (2000),
  "A deflated version of the conjugate gradient algorithm", with deflation
  space W (here the per-RHS recycle space U_j of Sec. 4.2).  This is the
  inner solver the CUDA path uses for the correction equation A~ g_j = r_j
  (Sec. 4.2.1, eq. resi); the paper's own inner solver is recycled MINRES,
  which reaches the same x_j.

Stopping rule shared by both Krylov solvers: iterate while the recursive
residual exceeds tol*||b_ref||; when it drops below, recompute the true
residual b - A x explicitly and stop only if that one is below too; else
restart from the true residual.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def dense_solve(A, B):
    A = A.toarray() if sp.issparse(A) else np.asarray(A)
    return np.linalg.solve(A, B)


def direct_solve(A, B):
    """x = A^-1 B by sparse LU (scipy SuperLU)."""
    lu = spla.splu(sp.csc_matrix(A))
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        return lu.solve(B)
    return np.column_stack([lu.solve(np.ascontiguousarray(B[:, c])) for c in range(B.shape[1])])


def banded_cholesky_solve(A, B, bw):
    """Solve with the Cholesky factor of the band (upper form) of SPD A."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    ab = np.zeros((bw + 1, n))
    for d in range(bw + 1):
        diag = A.diagonal(d)
        ab[bw - d, d:] = diag
    c = sla.cholesky_banded(ab, lower=False)
    return sla.cho_solve_banded((c, False), B)


def cg(A, b, tol, x0=None, maxit=100000, b_ref=None):
    """Plain CG on A x = b; returns (x, iterations, true relres)."""
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b if b_ref is None else b_ref)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    it = 0
    while True:
        if np.linalg.norm(r) <= tol * nb:
            break
        p = r.copy()
        rr = r @ r
        while it < maxit:
            q = A @ p
            alpha = rr / (p @ q)
            x += alpha * p
            r -= alpha * q
            it += 1
            rr_new = r @ r
            if np.sqrt(rr_new) <= tol * nb:
                break
            p = r + (rr_new / rr) * p
            rr = rr_new
        r = b - A @ x                       # explicit residual, restart if needed
        if it >= maxit:
            break
    return x, it, np.linalg.norm(b - A @ x) / nb


def deflated_cg(A, b, W, tol, b_ref_norm, x_init=None, maxit=100000, AW=None):
    """Deflated CG (Saad et al. 2000) on A x = b with deflation space W.

    Steps, per (re)start from x_{-1} with r_{-1} = b - A x_{-1}:
        x_0 = x_{-1} + W (W^T A W)^-1 W^T r_{-1};  r_0 = b - A x_0
        mu_0 = (W^T A W)^-1 (A W)^T r_0;           p_0 = r_0 - W mu_0
    and for j = 0, 1, ...:
        alpha_j = r_j^T r_j / p_j^T A p_j
        x_{j+1} = x_j + alpha_j p_j;  r_{j+1} = r_j - alpha_j A p_j
        beta_j  = r_{j+1}^T r_{j+1} / r_j^T r_j
        mu_{j+1} = (W^T A W)^-1 (A W)^T r_{j+1}
        p_{j+1} = r_{j+1} + beta_j p_j - W mu_{j+1}
    Stops when the explicitly recomputed ||b - A x|| <= tol * b_ref_norm.
    Returns (x, iterations, true residual norm / b_ref_norm)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x_init is None else np.array(x_init, dtype=np.float64)
    k = 0 if W is None else W.shape[1]
    if k:
        AW = A @ W if AW is None else AW
        GW = W.T @ AW
        cho = sla.cho_factor(GW)
    thresh = tol * b_ref_norm
    it = 0
    r = b - A @ x
    while np.linalg.norm(r) > thresh and it < maxit:
        if k:
            x = x + W @ sla.cho_solve(cho, W.T @ r)
            r = b - A @ x
            p = r - W @ sla.cho_solve(cho, AW.T @ r)
        else:
            p = r.copy()
        rr = r @ r
        while it < maxit and np.sqrt(rr) > thresh:
            q = A @ p
            alpha = rr / (p @ q)
            x = x + alpha * p
            r = r - alpha * q
            it += 1
            rr_new = r @ r
            beta = rr_new / rr
            rr = rr_new
            if np.sqrt(rr) <= thresh:
                break
            p = r + beta * p
            if k:
                p = p - W @ sla.cho_solve(cho, AW.T @ r)
        r = b - A @ x                       # explicit residual; loop restarts if too big
    return x, it, np.linalg.norm(b - A @ x) / b_ref_norm
