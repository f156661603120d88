"""Pins of the oracle's Algorithm 2 (Sec. 4.3): the ordered append against
its definition by brute force, the Galerkin check against an independent
least-squares route, the counting identity of Sec. 6 (ROM order = k_u + one
column per full-order solve) and the interpolation theorem of Sec. 3.4."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import basis, eigen, operator as op, rom, solvers
from synthetic.phantom import make_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")


def test_ordered_append_drops_dependent_columns():
    rng = np.random.default_rng(0)
    n = 200
    V0, _ = np.linalg.qr(rng.standard_normal((n, 5)))
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    X = np.column_stack([a, V0 @ rng.standard_normal(5), b, 2 * a - 3 * b + V0[:, 0],
                         a + 1e-10 * rng.standard_normal(n)])
    V, kept, ratios, Q = basis.ordered_append(V0, X, 1e-8)
    assert kept.tolist() == [True, False, True, False, False]
    assert V.shape[1] == 7 and len(Q) == 2
    assert np.linalg.norm(V.T @ V - np.eye(7)) < 1e-14
    # every candidate lies in the final span
    P = V @ (V.T @ X)
    assert np.linalg.norm(P - X) <= 1e-9 * np.linalg.norm(X)
    # ratios: a fresh random vector is far from the span, the copies are not
    assert ratios[0] > 0.9 and ratios[1] < 1e-14 and ratios[4] < 1e-9


def test_galerkin_check_equals_energy_norm_best_approximation():
    """x0 = V (V^T A V)^-1 V^T b minimises ||x - A^-1 b||_A over range(V):
    computed here instead by least squares with the Cholesky factor of A."""
    inp = make_workload("t2d_24")
    At, Bt, _ = op.assemble(inp, 1)
    A = At.toarray()
    rng = np.random.default_rng(1)
    V, _ = np.linalg.qr(rng.standard_normal((A.shape[0], 12)))
    b = Bt[:, 2]
    x0, r0, rel = basis.galerkin_check(At, V, b)
    L = sla.cholesky(A, lower=True)
    xs = np.linalg.solve(A, b)
    y, *_ = np.linalg.lstsq(L.T @ V, L.T @ xs, rcond=None)
    assert np.linalg.norm(x0 - V @ y) <= 1e-10 * np.linalg.norm(x0)
    assert np.isclose(rel, np.linalg.norm(b - A @ (V @ y)) / np.linalg.norm(b), rtol=1e-8)


def _run(name, order, tau):
    inp = make_workload(name)
    wl = inp["wl"]
    A0, Bt, Ct = op.assemble(inp, 0)
    B = np.hstack([Bt, Ct])
    _, U0 = eigen.smallest_eigenpairs(A0, wl.k_u)
    st = basis.seed(A0, B, U0, inp["tol"], tau=tau)
    As = {i: op.assemble(inp, i)[0] for i in range(1, wl.K + 1)}
    out = basis.solve_all(st, lambda i: As[i], range(1, wl.K + 1), B, inp["tol"],
                          order=order, tau=tau, keep_x=True)
    return inp, st, out, As, Bt, Ct


@pytest.mark.parametrize("name", ["t2d_24", "t3d_12"])
def test_sequential_algorithm2_invariants(name):
    inp, st, out, As, Bt, Ct = _run(name, "sequential", 1e-12)
    wl = inp["wl"]
    golden = json.load(open(GOLDEN))
    # Sec. 6: ROM order = k_u + number of full-order solves, each solve one column
    for e in ("experiment1", "experiment2"):
        assert golden[e]["rom_order"] == golden["k_u"] + golden[e]["full_order_solves"]
    n_solves = wl.nrhs + sum(o["iters"] > 0 for o in out)
    assert st.r == wl.k_u + n_solves
    assert all(o["appended"] == (o["iters"] > 0) for o in out)
    # every delivered solution meets its tolerance (explicit residual, dense check)
    for o in out:
        A = As[o["sample"]]
        b = np.hstack([Bt, Ct])[:, o["rhs"]]
        rel = np.linalg.norm(b - A @ o["x"]) / np.linalg.norm(b)
        assert rel <= inp["tol"][o["rhs"]] * 1.0000001
        # brute force: the check decision from a dense direct Galerkin solve
    assert np.linalg.norm(st.V.T @ st.V - np.eye(st.r)) < 1e-12
    # some right-hand sides at later samples need no iterations (Table 1 pattern)
    # or at least need fewer iterations than the seed solves did
    seed_its = np.mean([s["iters"] for s in st.stats[:wl.nrhs]])
    assert np.mean([o["iters"] for o in out]) < 0.8 * seed_its


def test_check_decisions_match_brute_force_replay():
    """Replay the sequential run: rebuild V column by column from the
    recorded decisions and recompute each check with dense direct solves."""
    inp, st, out, As, Bt, Ct = _run("t2d_24", "sequential", 1e-12)
    wl = inp["wl"]
    B = np.hstack([Bt, Ct])
    r = wl.k_u + wl.nrhs
    V = st.V[:, :r]
    for o in out:
        A = As[o["sample"]].toarray()
        b = B[:, o["rhs"]]
        G = V.T @ A @ V
        x0 = V @ np.linalg.solve(G, V.T @ b)
        rel0 = np.linalg.norm(b - A @ x0) / np.linalg.norm(b)
        assert np.isclose(rel0, o["relres0"], rtol=1e-6)
        assert (rel0 > inp["tol"][o["rhs"]]) == (o["iters"] > 0)
        if o["appended"]:
            r += 1
            V = st.V[:, :r]
    assert r == st.r


@pytest.mark.parametrize("order", ["sequential", "wave"])
def test_interpolation_theorem_at_sampled_points(order):
    """Sec. 3.4: Psi_r and grad Psi_r match at the sampled points.  With
    solutions at relres <= tol in range(V), the Galerkin error bound gives
    |Psi - Psi_r| <= tol^2 ||b~_s|| ||c~_d|| / lambda_min(A~)."""
    tau = 1e-12 if order == "sequential" else 1e-10
    inp, st, out, As, Bt, Ct = _run("t2d_24", order, tau)
    tol = inp["tol"].max()
    for i, A in As.items():
        P, J = rom.full_eval(A, Bt, Ct, inp["h"], inp["dmu"][i])
        Pr, Jr = rom.rom_eval(st.V, A, Bt, Ct, inp["h"], inp["dmu"][i])
        lmin = np.linalg.eigvalsh(A.toarray())[0]
        bound = tol ** 2 * np.outer(np.linalg.norm(Ct, axis=0), np.linalg.norm(Bt, axis=0)) / lmin
        assert np.all(np.abs(P - Pr) <= 10 * bound + 1e-12 * np.abs(P).max())  # rounding floor ~ kappa * eps
        assert np.linalg.norm(J - Jr) <= 1e-6 * np.linalg.norm(J)
        # the first-order Jacobian bound used by the GPU parity tests holds here
        from tests.gpu_common import jacobian_galerkin_bound
        lmin = np.linalg.eigvalsh(A.toarray())[0]
        bJ, Jb = jacobian_galerkin_bound(A, Bt, Ct, inp["h"], inp["dmu"][i], inp["tol"], tau, lmin)
        assert np.allclose(Jb, J, rtol=1e-12, atol=0)
        assert np.linalg.norm(J - Jr) <= bJ * np.linalg.norm(J)


def test_wave_order_appends_in_order_and_freezes_basis():
    inp, st, out, As, Bt, Ct = _run("t2d_24", "wave", 1e-8)
    wl = inp["wl"]
    kept = [o for o in out if o["appended"]]
    assert st.r == wl.k_u + wl.nrhs + len(kept)
    # all checks of a wave used the seed basis: relres0 of RHS j at sample 1
    # equals that of a fresh check with the seed basis
    r0 = wl.k_u + wl.nrhs
    V0 = st.V[:, :r0]
    B = np.hstack([Bt, Ct])
    for o in out[:3]:
        _, _, rel = basis.galerkin_check(As[o["sample"]], V0, B[:, o["rhs"]])
        assert np.isclose(rel, o["relres0"], rtol=1e-8)
    # a candidate is kept iff its new part exceeds tau; the corrections of one
    # wave are nearly low rank (Delta_i is diagonal on a small support), so
    # the later candidates of a wave carry less and less new information
    for o in out:
        if o["iters"] > 0:
            assert o["appended"] == (o["ratio"] > 1e-8)
    rat = [o["ratio"] for o in out if o["iters"] > 0]
    assert rat[-1] < 1e-2 * rat[0]


def test_private_recycle_space_cap_evicts_the_oldest_column():
    """U_j keeps at most k_cap columns: with k_cap = k_u + 2 and four
    appended columns for one right-hand side, X_0(:, j) goes first, then the
    older appended columns; U_0 is never evicted and the order is kept."""
    rng = np.random.default_rng(11)
    n, k_u = 30, 3
    U0 = rng.standard_normal((n, k_u))
    X0 = rng.standard_normal((n, 2))
    st = basis.BasisState(V=np.zeros((n, 0)), U0=U0, X0=X0, priv=[[X0[:, 0].copy()], [X0[:, 1].copy()]],
                          k_cap=k_u + 2)
    q = [rng.standard_normal(n) for _ in range(4)]
    st.push_private(0, q[0])
    assert np.array_equal(st.U(0), np.column_stack([U0, X0[:, 0], q[0]]))
    for c in q[1:]:
        st.push_private(0, c)
    assert np.array_equal(st.U(0), np.column_stack([U0, q[2], q[3]]))
    assert np.array_equal(st.U(1), np.column_stack([U0, X0[:, 1]]))     # other RHS untouched
