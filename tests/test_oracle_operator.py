"""Pins of the oracle's operator (Sec. 2.1, Sec. 3) against facts it does
not compute itself: a manufactured continuum solution, the constant
coefficient closed-form spectrum, the block structure stated in Sec. 3 and
the full-versus-Schur transfer function identity of Sec. 3.1."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import operator as op
from oracle import rom, solvers
from synthetic.phantom import make_workload

ROBIN_A = 1.0


def _grid_points(dims, h):
    Nx, Ny, Nz = dims
    g = lambda N: np.arange(1, N + 1) * h
    if Ny == 1:
        z, x = np.meshgrid(g(Nz), g(Nx), indexing="ij")
        return [x.ravel(), z.ravel()]
    z, y, x = np.meshgrid(g(Nz), g(Ny), g(Nx), indexing="ij")
    return [x.ravel(), y.ravel(), z.ravel()]


def _manufactured(dim, N):
    """Solve the full FD system for a manufactured solution, return max error.

    eta = sin(pi x) [sin(pi y)] zeta(z), zeta = 1 + z + z^2,
    D = 0.3 + 0.1 x z (+ 0.05 y), mu = 0.02 + 0.01 x.
    f = -div(D grad eta) + mu eta; Robin data g = eta + 2 A D d eta/d xi."""
    h = 1.0 / (N + 1)
    dims = (N, 1, N) if dim == 2 else (N, N, N)
    P = _grid_points(dims, h)
    x, z = P[0], P[-1]
    y = P[1] if dim == 3 else None

    def fields(x, y, z):
        sy = np.sin(np.pi * y) if y is not None else 1.0
        cy = np.cos(np.pi * y) if y is not None else 0.0
        zeta, dzeta, ddzeta = 1 + z + z * z, 1 + 2 * z, 2.0
        eta = np.sin(np.pi * x) * sy * zeta
        ex = np.pi * np.cos(np.pi * x) * sy * zeta
        exx = -np.pi ** 2 * eta
        ey = np.sin(np.pi * x) * np.pi * cy * zeta if y is not None else 0.0
        eyy = -np.pi ** 2 * eta if y is not None else 0.0
        ez = np.sin(np.pi * x) * sy * dzeta
        ezz = np.sin(np.pi * x) * sy * ddzeta
        D = 0.3 + 0.1 * x * z + (0.05 * y if y is not None else 0.0)
        Dx, Dy, Dz = 0.1 * z, (0.05 if y is not None else 0.0), 0.1 * x
        mu = 0.02 + 0.01 * x
        f = -(Dx * ex + D * exx + Dy * ey + D * eyy + Dz * ez + D * ezz) + mu * eta
        return eta, ez, D, mu, f

    eta, _, D, mu, f = fields(x, y, z)
    fs = op.full_system(dims, D, mu, h, ROBIN_A)
    Nx, Ny, _ = dims
    rhs = np.zeros(fs.nb + fs.n)
    rhs[fs.nb:] = h * h * f
    # Robin data on the two faces at the face points (x_i, y_j, 0) and (.., 1)
    fx = np.tile(np.arange(1, Nx + 1) * h, Ny)
    fy = np.repeat(np.arange(1, Ny + 1) * h, Nx) if dim == 3 else None
    for top, zb in ((False, 0.0), (True, 1.0)):
        e_b, ez_b, D_b, _, _ = fields(fx, fy, np.full(fx.shape, zb))
        dxi = ez_b if top else -ez_b                     # outward normal derivative
        g = e_b + 2 * ROBIN_A * D_b * dxi
        off = Nx * Ny if top else 0
        rhs[off:off + Nx * Ny] = g
    sol = spla.spsolve(fs.A.tocsc(), rhs)
    return np.max(np.abs(sol[fs.nb:] - eta))


@pytest.mark.parametrize("dim,Ns", [(2, (15, 31, 63)), (3, (7, 15, 31))])
def test_manufactured_solution_converges_first_order(dim, Ns):
    errs = [_manufactured(dim, N) for N in Ns]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    # first-order Robin rows dominate: error ~ O(h); a wrong sign, a missing
    # h^2 or a wrong face weight does not converge at all
    assert errs[-1] < 0.05, errs
    assert all(0.8 < r < 2.5 for r in rates), (errs, rates)


@pytest.mark.parametrize("dim,N", [(2, 10), (3, 6)])
def test_constant_coefficient_spectrum_is_kronecker_sum(dim, N):
    d0, m0 = 0.27, 0.013
    h = 1.0 / (N + 1)
    dims = (N, 1, N) if dim == 2 else (N, N, N)
    n = int(np.prod(dims))
    fs = op.full_system(dims, np.full(n, d0), np.full(n, m0), h, ROBIN_A)
    At = op.schur(fs).toarray()
    a = np.arange(1, N + 1)
    lam_dir = 2 - 2 * np.cos(a * np.pi / (N + 1))
    alpha = 2 * ROBIN_A * d0 / h
    dz = np.full(N, 2.0)
    dz[0] = dz[-1] = 1 + 1 / (1 + alpha)
    lam_rob, vz = sla.eigh_tridiagonal(dz, -np.ones(N - 1))
    if dim == 2:
        lam = (lam_dir[:, None] + lam_rob[None, :]).ravel()
    else:
        lam = (lam_dir[:, None, None] + lam_dir[None, :, None] + lam_rob[None, None, :]).ravel()
    lam = np.sort(d0 * lam + h * h * m0)
    got = np.linalg.eigvalsh(At)
    assert np.allclose(got, lam, rtol=0, atol=1e-12 * lam.max())
    # one explicit eigenvector: sine modes along the Dirichlet axes times a
    # Robin-axis eigenvector; index = i + Nx*(j + Ny*k)
    sx = np.sin(2 * a * np.pi / (N + 1))
    v = np.kron(vz[:, 1], sx) if dim == 2 else np.kron(vz[:, 1], np.kron(np.sin(a * np.pi / (N + 1)), sx))
    lam_v = d0 * ((2 - 2 * np.cos(2 * np.pi / (N + 1))) + (lam_dir[0] if dim == 3 else 0) + lam_rob[1]) + h * h * m0
    assert np.allclose(At @ v, lam_v * v, atol=1e-13)


@pytest.mark.parametrize("name", ["t2d_24", "t3d_12"])
def test_block_structure_and_spd(name):
    inp = make_workload(name)
    fs = op.full_system(inp["dims"], inp["D"], inp["mu"][1], inp["h"], inp["robin_A"])
    G, D1, D2, F = op.blocks(fs)
    # Sec. 3: G invertible diagonal; D1 at most one nonzero per row; D2 has D1^T's pattern
    assert (G - __import__("scipy.sparse", fromlist=["diags"]).diags(G.diagonal())).nnz == 0
    assert np.all(G.diagonal() > 1)
    assert np.all(np.diff(D1.indptr) == 1)
    assert ((D2 != 0).astype(int) != (D1.T != 0).astype(int)).nnz == 0
    At = op.schur(fs)
    assert abs(At - At.T).max() == 0.0                      # exactly symmetric
    sla.cholesky(At.toarray())                               # SPD
    # Delta = d A~ / d mu is diagonal h^2 (eq. sum): the only p-dependence
    fs2 = op.full_system(inp["dims"], inp["D"], inp["mu"][2], inp["h"], inp["robin_A"])
    dA = (op.schur(fs2) - At).tocoo()
    assert np.all(dA.row == dA.col)
    assert np.allclose(dA.diagonal(), inp["h"] ** 2 * (inp["mu"][2] - inp["mu"][1]), atol=1e-18)


@pytest.mark.parametrize("name", ["t2d_24", "t3d_12", "t2d_37"])
def test_full_system_transfer_function_equals_schur_form(name):
    """Psi(0) = C^T A^-1 B from the full nonsymmetric system equals
    C~^T A~^-1 B~ (Sec. 3.1), and C1^T G^-1 B1 = 0 (no co-located pairs)."""
    inp = make_workload(name)
    fs = op.full_system(inp["dims"], inp["D"], inp["mu"][1], inp["h"], inp["robin_A"])
    At = op.schur(fs)
    Bt, Ct, B1, C1 = op.effective_sources(fs, inp["src_ij"], inp["det_ij"])
    Bfull = np.vstack([B1, np.zeros((fs.n, B1.shape[1]))])
    Y = solvers.dense_solve(fs.A, Bfull)
    Psi_full = C1.T @ Y[:fs.nb]
    Psi, _ = rom.full_eval(At, Bt, Ct, inp["h"])
    assert np.linalg.norm(Psi_full - Psi) <= 1e-12 * np.linalg.norm(Psi)
    G, _, _, _ = op.blocks(fs)
    assert np.all(C1.T @ (B1 / G.diagonal()[:, None]) == 0)
    # effective sources are scaled identity columns at the face-adjacent nodes
    assert np.all((Bt != 0).sum(0) == 1) and np.all(Bt >= 0)
    assert np.all(np.nonzero(Bt)[0] == inp["src_nodes"])
    assert np.all(np.nonzero(Ct.T)[1] == inp["det_nodes"])
