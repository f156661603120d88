"""Pins of the oracle's transfer function, Jacobian and reduced model:
central finite differences of Psi (eq. newjac), source-detector reciprocity
(A~ symmetric, Sec. 3.3), exactness of the reduced model when range(V)
holds the primal and dual solutions (Theorem of Sec. 3.4) and with V = I."""
import numpy as np
import pytest

from oracle import operator as op, rom, solvers
from synthetic.phantom import make_workload, pals_mu


@pytest.mark.parametrize("name", ["t2d_24", "t3d_12"])
def test_jacobian_matches_central_differences(name):
    inp = make_workload(name)
    wl = inp["wl"]
    s = 1
    p = inp["params"][s]
    At, Bt, Ct = op.assemble(inp, s)
    _, J = rom.full_eval(At, Bt, Ct, inp["h"], inp["dmu"][s])

    def psi(pp):
        mu = pals_mu(pp, inp["X"], wl.mu_bg)
        A = op.schur_for_mu(inp, mu)
        return rom.full_eval(A, Bt, Ct, inp["h"])[0]

    for k in range(wl.nparam):
        d = 1e-6 * max(1.0, abs(p[k]))
        e = np.zeros_like(p); e[k] = d
        fd = (psi(p + e) - psi(p - e)) / (2 * d)
        scale = np.linalg.norm(J[k]) + 1e-30
        assert np.linalg.norm(fd - J[k]) <= 1e-5 * max(scale, 1e-3 * np.linalg.norm(J)), k
    assert np.linalg.norm(J) > 0


def test_reciprocity_of_transfer_function():
    inp = make_workload("t3d_12")
    At, Bt, Ct = op.assemble(inp, 2)
    X = solvers.direct_solve(At, Bt)
    Z = solvers.direct_solve(At, Ct)
    P_src = Ct.T @ X          # from source solutions
    P_det = Z.T @ Bt          # from detector solutions
    assert np.linalg.norm(P_src - P_det) <= 1e-12 * np.linalg.norm(P_src)
    assert np.all(P_src > 0)  # light from every source reaches every detector


def test_reduced_model_exact_when_basis_holds_solutions():
    inp = make_workload("t2d_24")
    At, Bt, Ct = op.assemble(inp, 1)
    X = solvers.direct_solve(At, Bt)
    Z = solvers.direct_solve(At, Ct)
    Psi, J = rom.full_eval(At, Bt, Ct, inp["h"], inp["dmu"][1], X=X, Z=Z)
    # a non-orthonormal basis of range([X, Z]) plus noise directions
    rng = np.random.default_rng(3)
    V = np.hstack([X, Z, rng.standard_normal((X.shape[0], 5))]) @ rng.standard_normal((X.shape[1] + Z.shape[1] + 5,) * 2)
    V, _ = np.linalg.qr(V)
    Pr, Jr = rom.rom_eval(V, At, Bt, Ct, inp["h"], inp["dmu"][1])
    assert np.linalg.norm(Pr - Psi) <= 1e-10 * np.linalg.norm(Psi)
    assert np.linalg.norm(Jr - J) <= 1e-8 * np.linalg.norm(J)
    # V = identity: the reduced model is the full model
    Pi, Ji = rom.rom_eval(np.eye(X.shape[0]), At, Bt, Ct, inp["h"], inp["dmu"][1])
    assert np.linalg.norm(Pi - Psi) <= 1e-12 * np.linalg.norm(Psi)
    assert np.linalg.norm(Ji - J) <= 1e-11 * np.linalg.norm(J)
    # a basis missing the solutions does not interpolate
    Vb, _ = np.linalg.qr(rng.standard_normal((X.shape[0], 20)))
    Pb, _ = rom.rom_eval(Vb, At, Bt, Ct, inp["h"])
    assert np.linalg.norm(Pb - Psi) > 1e-3 * np.linalg.norm(Psi)
