"""The paper's own inner solver and check (Sec. 4.1-4.2), restated in float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Minimum-residual check (Sec. 4.2.1 and the check of Algorithm 2):
    K~ = A~ V,  K~ = K R (thin QR),  U = V R^-1 (so A~ U = K, K^T K = I);
    z_j = U K^T b_j minimises ||b_j - A~ x|| over x in range(V) (eq. initialz);
    r_j = b_j - A~ z_j, recomputed explicitly here (in exact arithmetic it is
    (I - K K^T) b_j); V suffices for RHS j iff ||r_j|| / ||b_j|| <= tol_j.

Recycled MINRES on the correction equation A~ g_j = r_j (eq. resi) with a
recycle space U_j (Sec. 4.1, eqs. eq01 and SmallMin; Algorithm 2's inner
solve):
    A~ U_j = K~_j = K_j R_j (thin QR), U_j <- U_j R_j^-1 (A~ U_j = K_j);
    a Lanczos recurrence with the projected operator (I - K_j K_j^T) A~ from
    v_1 = (I - K_j K_j^T) r / xi, xi = ||(I - K_j K_j^T) r|| gives
        (I - K_j K_j^T) A~ V_m = V_{m+1} T_m   (T_m tridiagonal, (m+1) x m);
    y minimises ||xi e_1 - T_m y|| (MINRES: Givens QR of T_m, the iterate
    y_m = V_m y by short recurrences of direction vectors), and
        g = U_j K_j^T r + y_m - U_j K_j^T A~ y_m
    minimises ||r - A~ g|| over range([U_j, V_m]); ||r - A~ g|| = |phibar_m|,
    the MINRES residual estimate.  The first term vanishes when r is already
    orthogonal to range(K_j) (the case of eq. resi, where range(K_j) lies in
    range(K)).  Stop rule as in solvers.deflated_cg: iterate while
    |phibar| > tol ||b||, then recompute the residual explicitly and start a
    new cycle from it if it is still too large.

Per-RHS recycling only (Sec. 6.3, the comparison method of Table 2, after
Kilmer & de Sturler 2006): no global basis check; every system A~_i x = b_j
is solved by the same recycled MINRES with U_j = [U_0, X_0(:, j), earlier
new directions of RHS j], starting from the minimum-residual guess in
range(U_j); the new direction y_m goes into U_j only.

Parity: pinned by tests/test_oracle_minres.py -- the check equals a least
squares solve with A~ V; every MINRES iterate equals the minimiser of the
residual over range([U_j, Krylov space of the projected operator]) computed
by a dense least-squares solve; with U_j empty the iteration counts equal
scipy's MINRES on the same stopping level; the Table 2 direction (the
inner-outer method needs far fewer iterations than per-RHS recycling).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def recycle_basis(A, U):
    """(U R^-1, K) with A U = K R, K^T K = I (thin QR of A U); empty U gives
    empty arrays."""
    n = A.shape[0]
    if U is None or U.shape[1] == 0:
        return np.zeros((n, 0)), np.zeros((n, 0))
    K, R = np.linalg.qr(A @ U)
    Uh = sla.solve_triangular(R, U.T, trans="T", lower=False).T       # U R^-1
    return Uh, K


def mr_check(A, V, b):
    """Minimum-residual guess from range(V) and its explicit residual:
    (z, r, relres)."""
    if V.shape[1] == 0:
        return np.zeros_like(b), b.copy(), 1.0
    Uh, K = recycle_basis(A, V)
    z = Uh @ (K.T @ b)
    r = b - A @ z
    return z, r, np.linalg.norm(r) / np.linalg.norm(b)


def minres_cycle(A, r, Uh, K, thresh, maxit, trace=None):
    """One recycled MINRES cycle on A g = r (see the module docstring).
    Returns (g, iterations, |phibar| at exit).  `trace`, if a list, receives
    the iterate g after every iteration (for the tests)."""
    n = r.shape[0]
    k = K.shape[1]
    proj = (lambda w: w - K @ (K.T @ w)) if k else (lambda w: w)
    g0 = Uh @ (K.T @ r) if k else np.zeros(n)
    r1 = proj(r)
    xi = np.linalg.norm(r1)
    y = np.zeros(n)                      # y_m = V_m y_small, built by the recurrences
    if xi == 0.0:
        return g0, 0, 0.0
    v_prev = np.zeros(n)
    v = r1 / xi
    # Givens data of the two previous columns and the directions d_{k-1}, d_{k-2}
    c1, s1 = 1.0, 0.0                    # rotation k-1
    c2, s2 = 1.0, 0.0                    # rotation k-2
    d1 = np.zeros(n)
    d2 = np.zeros(n)
    phibar = xi
    it = 0
    beta_k = 0.0                         # T(k-1, k) of the current column (beta_k for k >= 2)
    while it < maxit and abs(phibar) > thresh:
        it += 1
        w = proj(A @ v)
        alpha = v @ w
        w = w - alpha * v - beta_k * v_prev
        beta_next = np.linalg.norm(w)
        # previous rotations applied to the new column [beta_k, alpha, beta_next]
        eps = s2 * beta_k
        dbar = c2 * beta_k
        delta = c1 * dbar + s1 * alpha
        gbar = -s1 * dbar + c1 * alpha
        gamma = np.hypot(gbar, beta_next)
        if gamma == 0.0:
            break
        c, s = gbar / gamma, beta_next / gamma
        tau = c * phibar
        phibar = -s * phibar
        d = (v - delta * d1 - eps * d2) / gamma
        y = y + tau * d
        d2, d1 = d1, d
        c2, s2, c1, s1 = c1, s1, c, s
        v_prev, v = v, (w / beta_next if beta_next > 0 else np.zeros(n))
        beta_k = beta_next
        if trace is not None:
            trace.append(g0 + y - (Uh @ (K.T @ (A @ y)) if k else 0.0))
        if beta_next == 0.0:
            break
    g = g0 + y - (Uh @ (K.T @ (A @ y)) if k else 0.0)
    return g, it, abs(phibar)


def recycled_minres(A, r, U, tol, b_ref_norm, maxit=100000):
    """Recycled MINRES on A g = r with recycle space U (columns, may be empty),
    cycles until the explicit residual ||r - A g|| <= tol b_ref_norm.
    Returns (g, iterations, relres ||r - A g|| / b_ref_norm)."""
    Uh, K = recycle_basis(A, U)
    thresh = tol * b_ref_norm
    g = np.zeros_like(r)
    res = r.copy()
    its = 0
    while np.linalg.norm(res) > thresh and its < maxit:
        dg, k_it, _ = minres_cycle(A, res, Uh, K, thresh, maxit - its)
        g = g + dg
        its += k_it
        res = r - A @ g                    # explicit residual; a new cycle if still too large
        if k_it == 0:
            break
    return g, its, np.linalg.norm(res) / b_ref_norm
