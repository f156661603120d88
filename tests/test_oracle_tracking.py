"""Pins of the oracle's diffusion-tracks-absorption operator
(oracle/operator.py: diffusion_of_mu, assemble_tracking, schur_derivative,
rhs_derivative) and of the product-rule Jacobians (oracle/rom.py:
full_eval_general, rom_eval_general), against facts that do not use the
derivative formulas: central differences of the assembled matrices, vectors
and transfer functions, the Hermite interpolation of Sec. 3.4 and the fixed-D
special case (eq. newjac)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import basis, eigen, operator as op, rom, solvers
from synthetic.phantom import make_workload, pals_dmu, pals_mu

MUS = 1.0        # reduced scattering mu_s'


def _at(inp, p):
    wl = inp["wl"]
    mu = pals_mu(p, inp["X"], wl.mu_bg)
    return mu, op.assemble_tracking(inp, mu, MUS)


def _near_faces(inp, s=1):
    """The parameters of sample s with the first anomaly moved next to the
    source face and the second next to the detector face, so that D changes
    at source and detector nodes (the terms dB~, dC~ are not zero there)."""
    wl = inp["wl"]
    d, h = wl.dim, inp["h"]
    p = np.array(inp["params"][s], dtype=np.float64).reshape(-1, d + 2)
    for a, (ij, z) in enumerate(((inp["src_ij"][0], 0.08), (inp["det_ij"][0], 0.92))):
        p[a, :d - 1] = np.asarray(ij[:d - 1], dtype=np.float64) * h      # over the first source / detector
        p[a, d - 1], p[a, d] = z, 0.14
    return p.ravel()


def _derivs(inp, p):
    """dA~_k, dB~_k, dC~_k of every parameter k at p (chain rule dD = -3 D^2 dmu)."""
    wl = inp["wl"]
    mu = pals_mu(p, inp["X"], wl.mu_bg)
    dmu = pals_dmu(p, inp["X"], wl.mu_bg)
    D = op.diffusion_of_mu(mu, MUS)
    dA, dB, dC = [], [], []
    for k in range(wl.nparam):
        dD = -3.0 * D * D * dmu[k]
        dA.append(op.schur_derivative(inp["dims"], D, dD, dmu[k], inp["h"], inp["robin_A"]))
        b, c = op.rhs_derivative(inp, D, dD)
        dB.append(b)
        dC.append(c)
    return dA, dB, dC


def test_tracking_operator_is_symmetric_positive_definite_and_reduces_to_fixed_d():
    inp = make_workload("t3d_12")
    mu = inp["mu"][1]
    At, Bt, Ct = op.assemble_tracking(inp, mu, MUS)
    assert abs(At - At.T).max() == 0.0
    np.linalg.cholesky(At.toarray())
    # at the seed point the workload's D is D(mu_0): the tracking operator is the fixed one
    A0, B0, C0 = op.assemble_tracking(inp, inp["mu"][0], MUS)
    F0, FB, FC = op.assemble(inp, 0)
    assert abs(A0 - F0).max() <= 1e-15 * abs(F0).max()
    assert np.array_equal(B0, FB) and np.array_equal(C0, FC)
    # elsewhere D differs, so the operators differ off the diagonal too
    F1, _, _ = op.assemble(inp, 1)
    diff = (At - F1).tocoo()
    off = diff.row != diff.col
    assert np.abs(diff.data[off]).max() > 0


@pytest.mark.parametrize("name", ["t2d_24", "t3d_12"])
def test_schur_and_rhs_derivatives_match_central_differences(name):
    inp = make_workload(name)
    wl = inp["wl"]
    p = _near_faces(inp)
    dA, dB, dC = _derivs(inp, p)
    assert max(np.abs(b).max() for b in dB) > 0 and max(np.abs(c).max() for c in dC) > 0
    checked = 0
    for k in range(wl.nparam):
        d = 1e-5 * max(1.0, abs(p[k]))
        e = np.zeros_like(p); e[k] = d
        _, (Ap, Bp, Cp) = _at(inp, p + e)
        _, (Am, Bm, Cm) = _at(inp, p - e)
        fdA = (Ap - Am) / (2 * d)
        scale = max(abs(dA[k]).max(), 1e-12)
        assert abs(fdA - dA[k]).max() <= 1e-6 * scale, k
        assert np.abs((Bp - Bm) / (2 * d) - dB[k]).max() <= 1e-6 * max(np.abs(dB[k]).max(), 1e-9), k
        assert np.abs((Cp - Cm) / (2 * d) - dC[k]).max() <= 1e-6 * max(np.abs(dC[k]).max(), 1e-9), k
        if abs(dA[k]).max() > 0:
            checked += 1
    assert checked >= wl.nparam // 2


def test_derivative_with_fixed_d_is_the_absorption_diagonal():
    inp = make_workload("t3d_12")
    s = 1
    D = inp["D"]
    dmu = inp["dmu"][s][3]
    M = op.schur_derivative(inp["dims"], D, np.zeros_like(D), dmu, inp["h"], inp["robin_A"])
    ref = sp.diags(inp["h"] ** 2 * dmu)
    assert abs(M - ref).max() == 0.0


@pytest.mark.parametrize("name", ["t2d_24", "t3d_12"])
def test_full_jacobian_matches_central_differences_of_psi(name):
    inp = make_workload(name)
    wl = inp["wl"]
    p = _near_faces(inp)
    _, (At, Bt, Ct) = _at(inp, p)
    dA, dB, dC = _derivs(inp, p)
    _, J = rom.full_eval_general(At, Bt, Ct, dA, dB, dC)

    def psi(pp):
        _, (A, B, C) = _at(inp, pp)
        return rom.full_eval_general(A, B, C)[0]

    for k in range(wl.nparam):
        d = 1e-6 * max(1.0, abs(p[k]))
        e = np.zeros_like(p); e[k] = d
        fd = (psi(p + e) - psi(p - e)) / (2 * d)
        assert np.linalg.norm(fd - J[k]) <= 1e-5 * max(np.linalg.norm(J[k]), 1e-3 * np.linalg.norm(J)), k
    # the tracking terms matter: the fixed-D Jacobian (eq. newjac alone) differs
    X = solvers.direct_solve(At, Bt)
    Z = solvers.direct_solve(At, Ct)
    J_fixed = np.stack([-(Z.T @ ((inp["h"] ** 2 * pals_dmu(p, inp["X"], wl.mu_bg)[k])[:, None] * X))
                        for k in range(wl.nparam)])
    assert np.linalg.norm(J_fixed - J) > 1e-3 * np.linalg.norm(J)


def test_reduced_jacobian_matches_central_differences_of_the_reduced_psi():
    """The product rule of rom_eval_general against differences of Psi_r(p)
    through a fixed random basis (no interpolation property involved)."""
    inp = make_workload("t2d_24")
    wl = inp["wl"]
    p = _near_faces(inp, 2)
    rng = np.random.default_rng(5)
    V, _ = np.linalg.qr(rng.standard_normal((wl.n, 17)))
    _, (At, Bt, Ct) = _at(inp, p)
    dA, dB, dC = _derivs(inp, p)
    _, Jr = rom.rom_eval_general(V, At, Bt, Ct, dA, dB, dC)

    def psi_r(pp):
        _, (A, B, C) = _at(inp, pp)
        return rom.rom_eval_general(V, A, B, C)[0]

    for k in range(wl.nparam):
        d = 1e-6 * max(1.0, abs(p[k]))
        e = np.zeros_like(p); e[k] = d
        fd = (psi_r(p + e) - psi_r(p - e)) / (2 * d)
        assert np.linalg.norm(fd - Jr[k]) <= 1e-5 * max(np.linalg.norm(Jr[k]), 1e-3 * np.linalg.norm(Jr)), k


def test_reduced_model_interpolates_value_and_jacobian_when_basis_holds_solutions():
    """Sec. 3.4: with A~(p)^-1 B~(p) and A~(p)^-1 C~(p) in range(V), Psi_r and
    its gradient equal Psi and its gradient at p, also when B~ and C~ follow p."""
    inp = make_workload("t3d_12")
    p = _near_faces(inp)
    _, (At, Bt, Ct) = _at(inp, p)
    dA, dB, dC = _derivs(inp, p)
    Psi, J = rom.full_eval_general(At, Bt, Ct, dA, dB, dC)
    X = solvers.direct_solve(At, Bt)
    Z = solvers.direct_solve(At, Ct)
    rng = np.random.default_rng(4)
    V, _ = np.linalg.qr(np.hstack([X, Z, rng.standard_normal((X.shape[0], 4))]))
    Pr, Jr = rom.rom_eval_general(V, At, Bt, Ct, dA, dB, dC)
    assert np.linalg.norm(Pr - Psi) <= 1e-10 * np.linalg.norm(Psi)
    assert np.linalg.norm(Jr - J) <= 1e-8 * np.linalg.norm(J)


def test_algorithm2_with_sample_dependent_rhs_delivers_every_tolerance():
    """solve_all with B~, C~ following the sample (a function of the sample):
    every delivered solution meets its tolerance for that sample's system."""
    inp = make_workload("t2d_24")
    wl = inp["wl"]
    sys = {i: op.assemble_tracking(inp, inp["mu"][i], MUS) for i in range(wl.K + 1)}
    A0, B0, C0 = sys[0]
    Bf0 = np.hstack([B0, C0])
    _, U0 = eigen.smallest_eigenpairs(A0, wl.k_u)
    st = basis.seed(A0, Bf0, U0, inp["tol"])
    out = basis.solve_all(st, lambda i: sys[i][0], range(1, wl.K + 1), lambda i: np.hstack(sys[i][1:]),
                          inp["tol"], keep_x=True)
    changed = 0
    for o in out:
        A, B, C = sys[o["sample"]]
        b = np.hstack([B, C])[:, o["rhs"]]
        assert np.linalg.norm(b - A @ o["x"]) <= inp["tol"][o["rhs"]] * np.linalg.norm(b) * 1.0001
        changed += not np.array_equal(b, Bf0[:, o["rhs"]])
    assert changed > 0              # some right-hand sides did move with the sample
