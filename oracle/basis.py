"""Algorithm 2 of the paper (Sec. 4.3, "Recycling and Global Basis
Construction") restated step by step in float64.

Seed (Algorithm 2, first three steps; Sec. 4.2.2 and Sec. 5.3):
    U_0 <- k_u eigenvectors of A~_0 for its smallest eigenvalues,
    X_0 solves A~_0 X_0 = B = [B~, C~],
    V <- basis of range([U_0, X_0]),  U_j <- [U_0, X_0(:, j)].
Outer loop over sample points i and right-hand sides j:
    check whether V represents x_j: Galerkin guess x0_j = V (V^T A~_i V)^-1 V^T b_j
      (the build's check; the paper's line uses the minimum-residual guess of
      eq. initialz -- both give a residual r_j with V^T-orthogonality to the
      respective test space), relres0_j = ||b_j - A~_i x0_j|| / ||b_j||
      recomputed explicitly;
    if relres0_j > tol_j: solve the correction equation A~_i g_j = r_j
      (eq. resi) with deflation space U_j, x_j = x0_j + g_j, and append the
      part of x_j not already in range(V) to V and to U_j (Sec. 4.2.2).
Order: `sequential` is the paper's order (V grows between right-hand sides);
`wave` freezes V for every (i, j) of the wave and appends the candidates
afterwards in ascending (i, j) order.

Append rule (the paper never drops a column; the drop test is a guard):
for each candidate x_c in order, w_c = (I - V V^T)^2 x_c against V and the
columns already accepted in this call; keep iff ||w_c|| / ||x_c|| > tau_rank;
the kept column is q_c = w_c / ||w_c||, appended to V and to U_j.
U_j keeps at most k_cap columns; when full, the oldest non-U_0 column goes.

Parity: pinned by brute-force decisions with dense direct solves on tiny
grids, the rank identity rank(V) = k_u + nrhs + #appends in sequential mode
(Sec. 6: 197 = 10 + 187), and the interpolation theorem of Sec. 3.4.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np
import scipy.linalg as sla

from . import minres
from .solvers import deflated_cg


@dataclass
class BasisState:
    V: np.ndarray                     # (n, r) orthonormal columns
    U0: np.ndarray                    # (n, k_u)
    X0: np.ndarray                    # (n, nrhs) seed solutions
    priv: list                        # per RHS: list of private recycle columns
    k_cap: int = 256
    stats: list = field(default_factory=list)

    @property
    def r(self):
        return self.V.shape[1]

    def U(self, j):
        cols = [self.U0] + [c[:, None] for c in self.priv[j]]
        return np.hstack(cols)

    def push_private(self, j, q):
        self.priv[j].append(q)
        while self.U0.shape[1] + len(self.priv[j]) > self.k_cap and self.priv[j]:
            self.priv[j].pop(0)


def ordered_append(V, X, tau):
    """Ordered rank-revealing append (see module docstring).
    Returns (V_new, kept mask, ratios, list of appended columns)."""
    V = np.array(V, dtype=np.float64).reshape(X.shape[0], -1)
    kept, ratios, Q = [], [], []
    for c in range(X.shape[1]):
        x = X[:, c]
        w = x.copy()
        for _ in range(2):
            if V.shape[1]:
                w = w - V @ (V.T @ w)
        ratio = np.linalg.norm(w) / np.linalg.norm(x)
        ratios.append(ratio)
        keep = ratio > tau
        kept.append(keep)
        if keep:
            q = w / np.linalg.norm(w)
            V = np.hstack([V, q[:, None]])
            Q.append(q)
    return V, np.array(kept), np.array(ratios), Q


def galerkin_check(A, V, b):
    """x0 = V (V^T A V)^-1 V^T b and its explicitly recomputed residual."""
    AV = A @ V
    G = V.T @ AV
    y = sla.cho_solve(sla.cho_factor(G), V.T @ b)
    x0 = V @ y
    r0 = b - A @ x0
    return x0, r0, np.linalg.norm(r0) / np.linalg.norm(b)


def solve_lane(A, b, tol, V, W, check="galerkin", inner="cg"):
    """Check, then (if needed) the inner solver on the correction equation:
    check "galerkin" (the build's default) or "mr" (the paper's
    minimum-residual guess, minres.mr_check); inner "cg" (deflated CG with
    deflation space W) or "minres" (the paper's recycled MINRES with recycle
    space W, minres.recycled_minres)."""
    bn = np.linalg.norm(b)
    if V.shape[1]:
        x0, r0, rel0 = galerkin_check(A, V, b) if check == "galerkin" else minres.mr_check(A, V, b)
    else:
        x0, r0, rel0 = np.zeros_like(b), b.copy(), 1.0
    if rel0 <= tol:
        return dict(x=x0, x0=x0, iters=0, relres0=rel0, relres=rel0, solved=False)
    if inner == "minres":
        g, its, _ = minres.recycled_minres(A, r0, W, tol, bn)
    else:
        g, its, _ = deflated_cg(A, r0, W, tol, bn)
    x = x0 + g
    rel = np.linalg.norm(b - A @ x) / bn
    return dict(x=x, x0=x0, iters=its, relres0=rel0, relres=rel, solved=True)


def seed(A0, Bfull, U0, tols, tau=1e-12, k_cap=256, inner="cg"):
    """Seed step of Algorithm 2: V = basis([U_0, X_0]), U_j = [U_0, X_0(:, j)].
    X_0(:, j) is computed with the Galerkin guess from range(U_0) and deflated
    CG with W = U_0, to relres tol_j."""
    n, nrhs = Bfull.shape
    V, _, _, _ = ordered_append(np.zeros((n, 0)), U0, 1e-12)
    X0 = np.zeros((n, nrhs))
    stats = []
    for j in range(nrhs):
        res = solve_lane(A0, Bfull[:, j], tols[j], V, U0, inner=inner)
        X0[:, j] = res["x"]
        stats.append(dict(sample=0, rhs=j, iters=res["iters"], relres0=res["relres0"],
                          relres=res["relres"], appended=True))
    V, kept, ratios, _ = ordered_append(V, X0, tau)
    st = BasisState(V=V, U0=U0.copy(), X0=X0, priv=[[X0[:, j].copy()] for j in range(nrhs)],
                    k_cap=k_cap)
    for j in range(nrhs):
        stats[j]["appended"] = bool(kept[j])
        stats[j]["ratio"] = float(ratios[j])
    st.stats.extend(stats)
    return st


def solve_all(st: BasisState, A_of, samples, Bfull, tols, order="sequential", tau=1e-12,
              keep_x=False, check="galerkin", inner="cg", wave_samples=0, wave_rhs=0):
    """Outer loop of Algorithm 2 over `samples` (A_of(i) gives A~_i); check
    and inner as in solve_lane (check="mr", inner="minres" is the paper's
    own form of Algorithm 2); wave order in waves of wave_samples samples x
    wave_rhs right-hand sides (0: all).  Bfull is the n x nrhs matrix
    [B~, C~], or a function of the sample giving it (B~ and C~ follow the
    sample when D tracks mu)."""
    samples = list(samples)
    B_of = Bfull if callable(Bfull) else (lambda i: Bfull)
    nrhs = B_of(samples[0]).shape[1]
    out = []
    if order == "sequential":
        for i in samples:
            A = A_of(i)
            for j in range(nrhs):
                res = solve_lane(A, B_of(i)[:, j], tols[j], st.V, st.U(j), check, inner)
                rec = dict(sample=i, rhs=j, iters=res["iters"], relres0=res["relres0"],
                           relres=res["relres"], appended=False, ratio=0.0)
                if res["solved"]:
                    V, kept, ratios, Q = ordered_append(st.V, res["x"][:, None], tau)
                    rec["ratio"] = float(ratios[0])
                    if kept[0]:
                        st.V = V
                        st.push_private(j, Q[0])
                        rec["appended"] = True
                if keep_x:
                    rec["x"] = res["x"]
                out.append(rec)
    elif order == "wave":
        # waves of `wave_samples` samples x `wave_rhs` consecutive RHS (0 = all):
        # V and every U_j are frozen within a wave; its candidates are appended
        # afterwards in ascending (sample, RHS) order
        ws = wave_samples if wave_samples > 0 else len(samples)
        wr = min(wave_rhs, nrhs) if wave_rhs > 0 else nrhs
        out = []
        for g0 in range(0, len(samples), ws):
            group = samples[g0:g0 + ws]
            for j0 in range(0, nrhs, wr):
                rhs = range(j0, min(j0 + wr, nrhs))
                V_wave = st.V
                U_wave = {j: st.U(j) for j in rhs}
                cands, recs = [], []
                for i in group:
                    A = A_of(i)
                    for j in rhs:
                        res = solve_lane(A, B_of(i)[:, j], tols[j], V_wave, U_wave[j], check, inner)
                        rec = dict(sample=i, rhs=j, iters=res["iters"], relres0=res["relres0"],
                                   relres=res["relres"], appended=False, ratio=0.0)
                        if keep_x:
                            rec["x"] = res["x"]
                        recs.append(rec)
                        if res["solved"]:
                            cands.append((len(recs) - 1, j, res["x"]))
                if cands:
                    X = np.column_stack([c[2] for c in cands])
                    V, kept, ratios, Q = ordered_append(st.V, X, tau)
                    st.V = V
                    qi = 0
                    for (ri, j, _), k, rt in zip(cands, kept, ratios):
                        recs[ri]["ratio"] = float(rt)
                        if k:
                            recs[ri]["appended"] = True
                            st.push_private(j, Q[qi])
                            qi += 1
                out.extend(recs)
        out.sort(key=lambda o: (o["sample"], o["rhs"]))
    else:
        raise ValueError(order)
    st.stats.extend(out)
    return out


def solve_all_per_rhs(st: BasisState, A_of, samples, Bfull, tols, tau=1e-12):
    """The comparison method of Sec. 6.3 (Table 2; recycling as in Kilmer & de
    Sturler 2006): no global basis.  For every sample i and RHS j the full
    system A~_i x = b_j is solved by recycled MINRES with the recycle space
    U_j of the state (U_0, X_0(:, j) and the earlier new directions of RHS j),
    from the minimum-residual guess in range(U_j); the part of x_j outside
    range(U_j) (normalised, if its relative size exceeds tau) joins U_j only.
    st.V is not used or changed.  Returns the per-(sample, RHS) records."""
    nrhs = Bfull.shape[1]
    out = []
    for i in samples:
        A = A_of(i)
        for j in range(nrhs):
            b = Bfull[:, j]
            bn = np.linalg.norm(b)
            W = st.U(j)
            z, r, rel0 = minres.mr_check(A, W, b)
            rec = dict(sample=i, rhs=j, iters=0, relres0=rel0, relres=rel0, appended=False)
            if rel0 > tols[j]:
                g, its, _ = minres.recycled_minres(A, r, W, tols[j], bn)
                x = z + g
                rec["iters"] = its
                rec["relres"] = np.linalg.norm(b - A @ x) / bn
                Q, _ = np.linalg.qr(W)
                w = x - Q @ (Q.T @ x)
                w = w - Q @ (Q.T @ w)
                if np.linalg.norm(w) > tau * np.linalg.norm(x):
                    st.push_private(j, w / np.linalg.norm(w))
                    rec["appended"] = True
            out.append(rec)
    return out
