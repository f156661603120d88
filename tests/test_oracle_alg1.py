"""Pins of the oracle's Algorithm 1 (truncated-SVD global basis, Sec. 4.2.2)
against facts that do not come from the oracle itself.

* Prescribed singular values: S = P diag(s) Q^T with orthonormal P, Q made
  here; the rank rule must count s_i > tau s_1 (capped by r_max) and range(V)
  must equal range(P[:, :r]) (principal angles ~ 0).
* Eckart-Young: ||S - V V^T S||_F^2 = sum_{i > r} s_i^2.
* Repeating columns changes no singular subspace: [S, S] gives the same V
  (singular values scaled by sqrt(2)).
* Interpolation (Theorem of Sec. 3.4): with every sampled solution in range(V)
  (r = full rank), the reduced model equals the full model at each sampled
  point.
"""
import numpy as np
import pytest

from oracle import alg1, operator as op, rom
from synthetic.phantom import make_workload


def _orth(rng, n, k):
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return Q


def _made(n=300, m=40, seed=3):
    rng = np.random.default_rng(seed)
    P = _orth(rng, n, m)
    Qm = _orth(rng, m, m)
    s = 10.0 ** (-np.arange(m) * 0.25)          # 1 .. 1e-9.75, distinct, well separated
    S = P @ np.diag(s) @ Qm.T
    return S, P, s


def _sin_angle(A, B):
    """Largest sine of the principal angles between range(A) and range(B) (orthonormal columns)."""
    if A.shape[1] == 0 and B.shape[1] == 0:
        return 0.0
    return float(np.linalg.norm(A - B @ (B.T @ A), 2))


@pytest.mark.parametrize("tau,r_max,expect", [(2e-3, 0, 11), (3e-6, 0, 23), (3e-6, 10, 10), (2.0, 0, 0)])
def test_rank_rule_and_subspace(tau, r_max, expect):
    S, P, s = _made()
    # split into "samples" of 8, 8, 8, 16 columns, as the blocks X_k
    blocks = [S[:, :8], S[:, 8:16], S[:, 16:24], S[:, 24:]]
    V, sigma = alg1.global_basis_svd(blocks, r_max, tau)
    # the count from the prescribed values (strictly above tau s_1), capped
    assert V.shape[1] == expect == min(int(np.sum(s > tau * s[0])), r_max if r_max > 0 else 10 ** 9)
    assert np.allclose(sigma, s, rtol=1e-8, atol=1e-14)
    if expect:
        assert _sin_angle(V, P[:, :expect]) < 1e-8
        assert np.allclose(V.T @ V, np.eye(expect), atol=1e-12)


def test_eckart_young_error():
    S, _, s = _made(seed=5)
    for r_max in (1, 5, 17):
        V, _ = alg1.global_basis_svd([S], r_max, 0.0)
        err2 = np.linalg.norm(S - V @ (V.T @ S), "fro") ** 2
        assert np.isclose(err2, np.sum(s[r_max:] ** 2), rtol=1e-6, atol=1e-24)


def test_repeated_columns_change_no_subspace():
    S, _, s = _made(seed=7)
    V1, s1 = alg1.global_basis_svd([S], 0, 1e-5)
    V2, s2 = alg1.global_basis_svd([S, S], 0, 1e-5)
    assert V1.shape == V2.shape
    assert _sin_angle(V1, V2) < 1e-8
    assert np.allclose(s2[: len(s1)], np.sqrt(2.0) * s1, rtol=1e-8)


def test_full_rank_basis_interpolates():
    """Theorem of Sec. 3.4: range(V) holds A~_k^-1 B~ and A~_k^-1 C~ -> Psi_r(p_k) = Psi(p_k)."""
    inp = make_workload("t2d_24")
    wl = inp["wl"]
    As, Bt, Ct = [], None, None
    for k in range(1, wl.K + 1):
        A, Bt, Ct = op.assemble(inp, k)
        As.append(A)
    blocks = alg1.snapshot_solves(As, np.hstack([Bt, Ct]))
    V, sigma = alg1.global_basis_svd(blocks, 0, 1e-13)
    assert V.shape[1] >= wl.nrhs
    for k, A in enumerate(As):
        P_r, _ = rom.rom_eval(V, A, Bt, Ct, inp["h"])
        P_f, _ = rom.full_eval(A, Bt, Ct, inp["h"])
        assert np.linalg.norm(P_r - P_f) <= 1e-9 * np.linalg.norm(P_f), k
    # a truncated basis no longer interpolates exactly
    Vt, _ = alg1.global_basis_svd(blocks, 3, 0.0)
    P_r, _ = rom.rom_eval(Vt, As[0], Bt, Ct, inp["h"])
    P_f, _ = rom.full_eval(As[0], Bt, Ct, inp["h"])
    assert np.linalg.norm(P_r - P_f) > 1e-6 * np.linalg.norm(P_f)
