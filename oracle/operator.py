"""Full-order finite-difference system and its symmetric Schur complement.

Restates Sec. 2.1 (eqs. ModelPDE1-4) and Sec. 3 (eq. block1, the Schur
complement A~ = F - D2 G^-1 D1, eqs. H, Sone, Stwo and the effective sources
B~ and receivers C~ of Sec. 3.1) in float64 with scipy.sparse.

Discretisation (Sec. 3: second-order centred differences inside, first-order
Robin rows on the boundary).  Readings of points the paper leaves open:
  * unknowns: N nodes per axis at x_i = i h, h = 1/(N+1); the lateral faces
    are homogeneous Dirichlet ghost layers (eq. ModelPDE3), the two z faces
    carry one Robin boundary unknown above / below each interior column
    (eq. ModelPDE2).  In 2D the axes are (x, z) and there is no y axis;
  * interior rows are scaled by h^2:
        sum_f w_f (eta_p - eta_q) + h^2 mu_p eta_p,
    with face weight w_f = (D_p + D_q)/2 between interior nodes and w_f = D_p
    on a face to a ghost or boundary node;
  * Robin row at boundary node b next to interior node p, with the outward
    normal derivative approximated by (eta_b - eta_p)/h:
        (1 + alpha_p) eta_b - alpha_p eta_p = s_b,   alpha_p = 2 A D_p / h;
  * ordering: boundary unknowns first (bottom face z=0, then top face z=1,
    each x fastest), then interior unknowns in natural order (Sec. 3).
Parity: pinned by the manufactured-solution convergence test, the
full-versus-Schur transfer-function identity, structural checks of G, D1,
D2 (Sec. 3 bullet list) and the constant-coefficient closed-form spectrum.

Diffusion tracking the absorption (an extension; Sec. 2.1 takes D as known
and fixed).  With the diffusion approximation's coefficient
    D(x; p) = 1 / (3 (mu(x; p) + mu_s')),
D changes with p wherever mu does, so A~, B~ and C~ all depend on p:
    * A~: every face weight and the Robin term D_p / (1 + alpha_p) of the
      Schur complement (eq. H and the block elimination of Sec. 3);
    * B~ = b D_p / (1 + alpha_p) e_p and C~ = c alpha_p / (1 + alpha_p) e_p
      at the face-adjacent node p of each source and detector (Sec. 3.1).
schur_derivative gives dA~ along a direction (dD, dmu) analytically:
    interior face (p, q):  w = (D_p + D_q)/2,      dw = (dD_p + dD_q)/2;
    ghost face of p:       w = D_p,                dw = dD_p;
    Robin face of p:       w = D_p/(1 + alpha_p),  dw = dD_p/(1 + alpha_p)^2;
    (dA~)_pq = -dw on interior faces, (dA~)_pp = sum of the dw of p's faces
    + h^2 dmu_p; rhs_derivative gives dB~ and dC~ (d/dD of D/(1+alpha) and of
    alpha/(1+alpha) = (2A/h)/(1+alpha)^2).  With dD = -3 D^2 dmu the chain
    rule through D(mu).  Pinned by central differences of the assembled
    matrices and vectors (tests/test_oracle_tracking.py).
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np
import scipy.sparse as sp


@dataclass
class FullSystem:
    A: sp.csr_matrix          # full nonsymmetric system, boundary-first ordering
    nb: int                   # number of Robin boundary unknowns
    n: int                    # number of interior unknowns
    dims: tuple


def _interior_index(dims):
    Nx, Ny, Nz = dims
    k, j, i = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    return i.ravel(), j.ravel(), k.ravel()


def full_system(dims, D, mu, h, robin_A) -> FullSystem:
    """Assemble the full FD system of Sec. 2.1 / eq. block1 at omega = 0."""
    Nx, Ny, Nz = dims
    n = Nx * Ny * Nz
    nface = Nx * Ny
    nb = 2 * nface
    D = np.asarray(D, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    i, j, k = _interior_index(dims)
    p = i + Nx * (j + Ny * k)
    rows, cols, vals = [], [], []

    def add(r, c, v):
        rows.append(np.asarray(r)); cols.append(np.asarray(c)); vals.append(np.asarray(v, dtype=np.float64))

    diag = h * h * mu[p]
    axes = [(i, Nx, 1)]
    if Ny > 1:
        axes.append((j, Ny, Nx))
    # lateral (Dirichlet) axes: interior neighbour or ghost with weight D_p
    for coord, extent, stride in axes:
        for step in (-1, 1):
            has = (coord + step >= 0) & (coord + step < extent)
            q = p + step * stride
            w = np.where(has, 0.5 * (D[p] + D[np.where(has, q, p)]), D[p])
            diag = diag + w
            add(nb + p[has], nb + q[has], -w[has])
    # Robin axis z: interior neighbour, or the boundary unknown on that face
    face = i + Nx * j
    for step in (-1, 1):
        has = (k + step >= 0) & (k + step < Nz)
        q = p + step * Nx * Ny
        w = np.where(has, 0.5 * (D[p] + D[np.where(has, q, p)]), D[p])
        diag = diag + w
        add(nb + p[has], nb + q[has], -w[has])
        bnd = ~has
        b = face[bnd] + (0 if step < 0 else nface)
        add(nb + p[bnd], b, -w[bnd])
        alpha = 2.0 * robin_A * D[p[bnd]] / h
        add(b, b, 1.0 + alpha)
        add(b, nb + p[bnd], -alpha)
    add(nb + p, nb + p, diag)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nb + n, nb + n)).tocsr()
    A.sum_duplicates()
    return FullSystem(A=A, nb=nb, n=n, dims=tuple(dims))


def blocks(fs: FullSystem):
    """Split the full system into G, D1, D2, F (eq. block1)."""
    A, nb = fs.A, fs.nb
    G = A[:nb, :nb].tocsr()
    D1 = A[:nb, nb:].tocsr()
    D2 = A[nb:, :nb].tocsr()
    F = A[nb:, nb:].tocsr()
    return G, D1, D2, F


def schur(fs: FullSystem):
    """A~ = F - D2 G^-1 D1 (Sec. 3, SPD at omega = 0)."""
    G, D1, D2, F = blocks(fs)
    ginv = sp.diags(1.0 / G.diagonal())
    At = (F - D2 @ ginv @ D1).tocsr()
    At.sum_duplicates()
    At.eliminate_zeros()
    return At


def boundary_columns(fs: FullSystem, face_ij, top: bool):
    """Columns of the identity on the Robin boundary unknowns at face points
    (1-based (i, j) lattice coordinates): the B_1 / C_1 blocks of Sec. 3.1."""
    Nx, Ny, _ = fs.dims
    nface = Nx * Ny
    M = np.zeros((fs.nb, len(face_ij)))
    for c, (ii, jj) in enumerate(face_ij):
        M[(ii - 1) + Nx * (jj - 1) + (nface if top else 0), c] = 1.0
    return M


def effective_sources(fs: FullSystem, src_ij, det_ij):
    """B~ = -D2 G^-1 B1 and C~ = -D1^T G^-1 C1 (Sec. 3.1).

    The signs follow from eliminating the boundary unknowns from
    A [y1; y2] = [B1; 0]: (F - D2 G^-1 D1) y2 = -D2 G^-1 B1 and
    Psi = C1^T y1 = -C1^T G^-1 D1 y2 (C1^T G^-1 B1 = 0 because sources and
    detectors are not co-located).  Both come out non-negative."""
    G, D1, D2, F = blocks(fs)
    ginv = sp.diags(1.0 / G.diagonal())
    B1 = boundary_columns(fs, src_ij, top=False)
    C1 = boundary_columns(fs, det_ij, top=True)
    Bt = -(D2 @ ginv @ B1)
    Ct = -(D1.T @ ginv @ C1)
    return np.asarray(Bt), np.asarray(Ct), B1, C1


def assemble(inp, s):
    """Convenience: A~ at sample s of a synthetic workload dict, and B~, C~."""
    fs = full_system(inp["dims"], inp["D"], inp["mu"][s], inp["h"], inp["robin_A"])
    At = schur(fs)
    Bt, Ct, _, _ = effective_sources(fs, inp["src_ij"], inp["det_ij"])
    return At, Bt, Ct


def schur_for_mu(inp, mu):
    fs = full_system(inp["dims"], inp["D"], mu, inp["h"], inp["robin_A"])
    return schur(fs)


# ------------------------------------------------- diffusion tracking mu
def diffusion_of_mu(mu, mu_s_prime):
    """D = 1 / (3 (mu + mu_s')): the diffusion coefficient of the diffusion
    approximation for absorption mu and reduced scattering mu_s'."""
    return 1.0 / (3.0 * (np.asarray(mu, dtype=np.float64) + mu_s_prime))


def assemble_tracking(inp, mu, mu_s_prime):
    """A~, B~, C~ at absorption mu with D = D(mu) (every coefficient of the
    full system of Sec. 2.1 follows the sample)."""
    D = diffusion_of_mu(mu, mu_s_prime)
    fs = full_system(inp["dims"], D, mu, inp["h"], inp["robin_A"])
    At = schur(fs)
    Bt, Ct, _, _ = effective_sources(fs, inp["src_ij"], inp["det_ij"])
    return At, Bt, Ct


def schur_derivative(dims, D, dD, dmu, h, robin_A):
    """dA~ (sparse, n x n) when D changes by dD and mu by dmu (module
    docstring): the face weights of A~ at D differentiated face by face."""
    Nx, Ny, Nz = dims
    n = Nx * Ny * Nz
    D = np.asarray(D, dtype=np.float64)
    dD = np.asarray(dD, dtype=np.float64)
    i, j, k = _interior_index(dims)
    p = i + Nx * (j + Ny * k)
    rows, cols, vals = [], [], []
    ddiag = h * h * np.asarray(dmu, dtype=np.float64)[p]
    axes = [(i, Nx, 1)]
    if Ny > 1:
        axes.append((j, Ny, Nx))
    for coord, extent, stride in axes:                 # Dirichlet axes: interior face or ghost face
        for step in (-1, 1):
            has = (coord + step >= 0) & (coord + step < extent)
            q = np.where(has, p + step * stride, p)
            dw = np.where(has, 0.5 * (dD[p] + dD[q]), dD[p])
            ddiag = ddiag + dw
            rows.append(p[has]); cols.append(q[has]); vals.append(-dw[has])
    for step in (-1, 1):                               # Robin axis: interior face or eliminated Robin face
        has = (k + step >= 0) & (k + step < Nz)
        q = np.where(has, p + step * Nx * Ny, p)
        alpha = 2.0 * robin_A * D[p] / h
        dw = np.where(has, 0.5 * (dD[p] + dD[q]), dD[p] / (1.0 + alpha) ** 2)
        ddiag = ddiag + dw
        rows.append(p[has]); cols.append(q[has]); vals.append(-dw[has])
    rows.append(p); cols.append(p); vals.append(ddiag)
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    M.sum_duplicates()
    return M


def rhs_derivative(inp, D, dD):
    """(dB~, dC~) when D changes by dD: the Robin elimination's source weight
    D_p/(1 + alpha_p) and detector weight alpha_p/(1 + alpha_p) at each
    face-adjacent node, differentiated in D_p (unit source / detector
    strengths, as in effective_sources)."""
    Nx, Ny, Nz = inp["dims"]
    n = Nx * Ny * Nz
    h, A = inp["h"], inp["robin_A"]
    D = np.asarray(D, dtype=np.float64)
    dD = np.asarray(dD, dtype=np.float64)

    def cols(face_ij, top):
        out = np.zeros((n, len(face_ij)))
        for c, (ii, jj) in enumerate(face_ij):
            node = (ii - 1) + Nx * ((jj - 1) + Ny * ((Nz - 1) if top else 0))
            alpha = 2.0 * A * D[node] / h
            dwt = (2.0 * A / h) / (1.0 + alpha) ** 2 if top else 1.0 / (1.0 + alpha) ** 2
            out[node, c] = dwt * dD[node]
        return out

    return cols(inp["src_ij"], False), cols(inp["det_ij"], True)
