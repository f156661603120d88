"""Seeded synthetic phantoms for the diffuse-optical-tomography forward problem.

The paper (Sec. 2.1) parametrises the unknown absorption mu(x; p) with
parametric level sets built from compactly supported radial basis functions
(Sec. 6).  The exact phantoms of its experiments are not published, so this
module generates stand-ins with the structure the experiments describe:

* level-set anomalies, one Gaussian bump per anomaly:
      phi_k(x) = exp(-|x - c_k|^2 / w_k^2) - 1/2,
      mu(x; p) = mu_bg + sum_k (m_k - mu_bg) * H(phi_k(x)),
  with H a C1 smoothed Heaviside that is exactly 0 for s <= -eps and exactly
  1 for s >= eps, so mu - mu_bg and every d mu / d p_k have finite support;
* per-anomaly parameters (c_k in R^d, w_k, m_k): d + 2 per anomaly, i.e. the
  paper's four parameters per basis function in 2D;
* a diffusion field fixed at the seed point, D = 1 / (3 (mu(x; p0) + mu_s')),
  held constant over the sample points (Sec. 2.1 takes D as known);
* sample points p_1..p_K obtained by jittering p0, standing in for the first
  parameter vectors an optimiser would produce (Sec. 3.4, Algorithm 1);
* sources on the z = 0 face and detectors on the z = 1 face on an even
  lattice, never co-located (Sec. 3.1).

Grid convention: N unknown nodes per axis at x_i = i h, i = 1..N, h = 1/(N+1).
In 2D the unknowns are (x, z) with z the Robin axis; the linear node index is
i + Nx*(j + Ny*k) with (Nx, Ny, Nz) = (N, 1, N) in 2D and (N, N, N) in 3D.
Random draws use numpy's PCG64 generator seeded per workload.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import numpy as np

H_EPS = 0.15          # half-width of the smoothed Heaviside, in level-set units


@dataclass(frozen=True)
class Workload:
    name: str
    dim: int                  # 2 or 3
    N: int                    # interior nodes per axis
    n_anom: int               # number of level-set anomalies
    src_lattice: tuple        # sources on the z=0 face: (count along x, count along y)
    det_lattice: tuple        # detectors on the z=1 face
    K: int                    # sample points p_1..p_K (p_0 is the seed point)
    tol: tuple = (1e-8,)      # per-RHS tolerance pattern, cycled over RHS index
    mu_anom: float | None = None   # fixed anomaly absorption, else U[0.02, 0.05]
    seed: int = 0
    mu_bg: float = 0.01
    mu_s_prime: float = 1.0
    robin_A: float = 1.0
    k_u: int = 10             # seed eigenvectors (Sec. 4.2)

    @property
    def dims(self):
        return (self.N, 1, self.N) if self.dim == 2 else (self.N, self.N, self.N)

    @property
    def n(self):
        Nx, Ny, Nz = self.dims
        return Nx * Ny * Nz

    @property
    def h(self):
        return 1.0 / (self.N + 1)

    @property
    def nsrc(self):
        return self.src_lattice[0] * self.src_lattice[1]

    @property
    def ndet(self):
        return self.det_lattice[0] * self.det_lattice[1]

    @property
    def nrhs(self):
        return self.nsrc + self.ndet

    @property
    def nparam(self):
        return self.n_anom * (self.dim + 2)


WORKLOADS = {
    # 2D 64x64, 16 + 16, 3 samples, FP64 plain recycled CG to relres 1e-10
    "c1_2d64": Workload("c1_2d64", 2, 64, 2, (16, 1), (16, 1), 3, (1e-10,), 0.03),
    # 3D 64^3, 32 + 32, 5 samples, tol 1e-8
    "c2_3d64": Workload("c2_3d64", 3, 64, 4, (8, 4), (8, 4), 5, (1e-8,)),
    # 3D 128^3, 64 + 64, 10 samples, tolerances alternating 1e-8 / 1e-6
    "c3_3d128": Workload("c3_3d128", 3, 128, 4, (8, 8), (8, 8), 10, (1e-8, 1e-6)),
    # 3D 128^3 learned augmentation: 64 + 64, 10 samples, tol 1e-8; the
    # network trains on plain-method solves at training_params phantoms
    "c4_3d128": Workload("c4_3d128", 3, 128, 4, (8, 8), (8, 8), 10, (1e-8,)),
    # 3D 192^3, 128 + 128, 20 samples, 8 anomalies
    "c5_3d192": Workload("c5_3d192", 3, 192, 8, (16, 8), (16, 8), 20, (1e-8,)),
    # the paper's experiment shape: 2D 201^2, 32 + 32, K* = 3, tol 1e-7 (Sec. 6)
    "paper_2d201": Workload("paper_2d201", 2, 201, 3, (32, 1), (32, 1), 3, (1e-7,)),
    # small cases for parity tests: several tiles and ragged tails
    "t2d_24": Workload("t2d_24", 2, 24, 2, (4, 1), (4, 1), 2, (1e-10,), 0.03, k_u=6),
    "t2d_37": Workload("t2d_37", 2, 37, 2, (6, 1), (5, 1), 3, (1e-9,), k_u=10),
    "t3d_12": Workload("t3d_12", 3, 12, 2, (2, 2), (2, 2), 2, (1e-10,), k_u=10),
    "t3d_21": Workload("t3d_21", 3, 21, 3, (3, 2), (2, 3), 3, (1e-8, 1e-6), k_u=10),
    "t3d_33": Workload("t3d_33", 3, 33, 4, (4, 4), (4, 4), 3, (1e-8,), k_u=10),
    "t3d_32": Workload("t3d_32", 3, 32, 3, (4, 2), (3, 3), 3, (1e-8, 1e-6), k_u=10),
    "t2d_40": Workload("t2d_40", 2, 40, 2, (7, 1), (6, 1), 3, (1e-9,), k_u=10),
    # 2D 48^2, 12 + 12, 2 samples: the iteration pattern of the paper's Table 2 at a small size
    "t2d_48": Workload("t2d_48", 2, 48, 2, (12, 1), (12, 1), 2, (1e-10,), 0.03, k_u=10),
    # 16^3: the plane-streaming stencil with a ragged y-tile (64-row tile, 16 rows)
    "t3d_16": Workload("t3d_16", 3, 16, 2, (2, 2), (2, 2), 3, (1e-8,), k_u=10),
}


def smooth_heaviside(s, eps=H_EPS):
    """C1 Heaviside: 0 below -eps, 1 above eps, 1/2 (1 + s/eps + sin(pi s/eps)/pi) between."""
    s = np.asarray(s, dtype=np.float64)
    t = np.clip(s / eps, -1.0, 1.0)
    mid = 0.5 * (1.0 + t + np.sin(np.pi * t) / np.pi)
    return np.where(s <= -eps, 0.0, np.where(s >= eps, 1.0, mid))


def smooth_heaviside_deriv(s, eps=H_EPS):
    s = np.asarray(s, dtype=np.float64)
    inside = np.abs(s) < eps
    return np.where(inside, (1.0 + np.cos(np.pi * s / eps)) / (2.0 * eps), 0.0)


def node_coords(wl: Workload):
    """(n, d) coordinates of the unknown nodes in linear-index order."""
    N, h = wl.N, wl.h
    g = np.arange(1, N + 1, dtype=np.float64) * h
    if wl.dim == 2:
        z, x = np.meshgrid(g, g, indexing="ij")          # index = i + N*k
        return np.stack([x.ravel(), z.ravel()], axis=1)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")       # index = i + N*(j + N*k)
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def node_grid(wl: Workload):
    """The `grid` argument of pals_mu / pals_dmu for node_coords(wl)."""
    return (wl.N, wl.h, wl.dim)


def _split(p, d):
    p = np.asarray(p, dtype=np.float64).reshape(-1, d + 2)
    return p[:, :d], p[:, d], p[:, d + 1]


def _support(X, c, w, grid=None):
    """Indices (ascending) of the points where phi = exp(-|x - c|^2 / w^2) - 1/2
    > -H_EPS, the only ones where an anomaly contributes (H and H' vanish
    elsewhere): a ball of radius w sqrt(ln(1 / (1/2 - H_EPS))), found by a
    per-axis box test.  grid = (N, h, d) says that X is the node grid of
    node_coords (coordinate i h, i = 1..N, along each axis, x fastest); the
    box test then runs only on the index box around the ball (one node wider
    on every side), which gives the same set."""
    R2 = w * w * np.log(1.0 / (0.5 - H_EPS))
    R = np.sqrt(R2) * (1.0 + 1e-12)
    if grid is None:
        box = np.abs(X[:, 0] - c[0]) < R
        for a in range(1, X.shape[1]):
            box &= np.abs(X[:, a] - c[a]) < R
        return np.nonzero(box)[0]
    N, h, d = grid
    rng = []
    for a in range(d):
        lo = max(1, int(np.floor((c[a] - R) / h)) - 1)
        hi = min(N, int(np.ceil((c[a] + R) / h)) + 1)
        if lo > hi:
            return np.zeros(0, dtype=np.int64)
        rng.append(np.arange(lo - 1, hi, dtype=np.int64))          # 0-based node index along the axis
    if d == 2:
        ix, iz = rng
        cand = (ix[None, :] + N * iz[:, None]).ravel()
    else:
        ix, iy, iz = rng
        cand = (ix[None, None, :] + N * (iy[None, :, None] + N * iz[:, None, None])).ravel()
    Xc = X[cand]
    box = np.abs(Xc[:, 0] - c[0]) < R
    for a in range(1, d):
        box &= np.abs(Xc[:, a] - c[a]) < R
    return cand[box]


def pals_mu(p, X, mu_bg, grid=None):
    """Absorption at points X (n, d) for parameter vector p (n_anom*(d+2));
    grid: see _support (a faster route on the node grid, same values)."""
    d = X.shape[1]
    c, w, m = _split(p, d)
    mu = np.full(X.shape[0], mu_bg, dtype=np.float64)
    for k in range(c.shape[0]):
        idx = _support(X, c[k], w[k], grid)
        r2 = np.sum((X[idx] - c[k]) ** 2, axis=1)
        phi = np.exp(-r2 / w[k] ** 2) - 0.5
        mu[idx] += (m[k] - mu_bg) * smooth_heaviside(phi)
    return mu


def pals_dmu(p, X, mu_bg, grid=None):
    """Analytic d mu / d p_k at points X: array (nparam, n); grid as in pals_mu."""
    d = X.shape[1]
    c, w, m = _split(p, d)
    out = np.zeros((c.shape[0] * (d + 2), X.shape[0]), dtype=np.float64)
    for k in range(c.shape[0]):
        idx = _support(X, c[k], w[k], grid)
        diff = X[idx] - c[k]
        r2 = np.sum(diff ** 2, axis=1)
        E = np.exp(-r2 / w[k] ** 2)
        phi = E - 0.5
        Hp = smooth_heaviside_deriv(phi)
        amp = m[k] - mu_bg
        base = k * (d + 2)
        for a in range(d):
            out[base + a, idx] = amp * Hp * E * 2.0 * diff[:, a] / w[k] ** 2
        out[base + d, idx] = amp * Hp * E * 2.0 * r2 / w[k] ** 3
        out[base + d + 1, idx] = smooth_heaviside(phi)
    return out


def seed_params(wl: Workload, rng):
    d = wl.dim
    p = np.zeros((wl.n_anom, d + 2))
    p[:, :d] = rng.uniform(0.15, 0.85, size=(wl.n_anom, d))
    p[:, d] = rng.uniform(0.05, 0.15, size=wl.n_anom)
    if wl.mu_anom is not None:
        p[:, d + 1] = wl.mu_anom
    else:
        p[:, d + 1] = rng.uniform(0.02, 0.05, size=wl.n_anom)
    return p.ravel()


def sample_params(wl: Workload, p0, rng, count):
    """Jittered parameter points around p0 (centres N(0, 0.02^2) clipped to
    [0.1, 0.9]; widths and anomaly absorptions scaled by 1 + U[-0.1, 0.1])."""
    d = wl.dim
    out = []
    for _ in range(count):
        q = np.array(p0, dtype=np.float64).reshape(-1, d + 2).copy()
        q[:, :d] = np.clip(q[:, :d] + rng.normal(0.0, 0.02, size=q[:, :d].shape), 0.1, 0.9)
        q[:, d] *= 1.0 + rng.uniform(-0.1, 0.1, size=q.shape[0])
        q[:, d + 1] *= 1.0 + rng.uniform(-0.1, 0.1, size=q.shape[0])
        out.append(q.ravel())
    return np.array(out)


def face_lattice(N, counts):
    """1-based in-face indices of an evenly spaced lattice of `counts` points."""
    return np.array([1 + int((a + 0.5) * N / counts) for a in range(counts)], dtype=np.int64)


def face_nodes(wl: Workload, lattice, top: bool):
    """Linear indices of the unknown nodes adjacent to the z=0 (top=False) or
    z=1 (top=True) face under a lattice of face points, in lattice order
    (x fastest).  Also returns the (i, j) face coordinates (1-based)."""
    Nx, Ny, Nz = wl.dims
    ix = face_lattice(Nx, lattice[0])
    iy = face_lattice(Ny, lattice[1]) if wl.dim == 3 else np.array([1])
    k = Nz if top else 1
    ij, nodes = [], []
    for j in iy:
        for i in ix:
            ij.append((i, j))
            nodes.append((i - 1) + Nx * ((j - 1) + Ny * (k - 1)))
    return np.array(nodes, dtype=np.int64), np.array(ij, dtype=np.int64)


def rhs_tolerances(wl: Workload):
    t = np.array(wl.tol, dtype=np.float64)
    return np.array([t[j % t.size] for j in range(wl.nrhs)], dtype=np.float64)


def make_workload(spec, K=None, seed=None, with_dmu=True):
    """Build every input of a workload.

    Returns a dict with: wl, dims, h, n, X (coords) [only for small n], params
    (K+1, nparam) with row 0 the seed point p0, mu (K+1, n), D (n), dmu (K+1,
    nparam, n) or None, src_nodes / det_nodes (interior node indices next to
    the faces), src_ij / det_ij (face coordinates), tol (nrhs,)."""
    wl = WORKLOADS[spec] if isinstance(spec, str) else spec
    if K is not None or seed is not None:
        wl = replace(wl, K=wl.K if K is None else K, seed=wl.seed if seed is None else seed)
    rng = np.random.default_rng(wl.seed)
    p0 = seed_params(wl, rng)
    ps = np.vstack([p0[None, :], sample_params(wl, p0, rng, wl.K)])
    X = node_coords(wl)
    grid = node_grid(wl)
    mu = np.stack([pals_mu(p, X, wl.mu_bg, grid) for p in ps])
    D = 1.0 / (3.0 * (mu[0] + wl.mu_s_prime))
    dmu = np.stack([pals_dmu(p, X, wl.mu_bg, grid) for p in ps]) if with_dmu else None
    src_nodes, src_ij = face_nodes(wl, wl.src_lattice, top=False)
    det_nodes, det_ij = face_nodes(wl, wl.det_lattice, top=True)
    return dict(wl=wl, dims=wl.dims, h=wl.h, n=wl.n, X=X, params=ps, mu=mu, D=D,
                dmu=dmu, src_nodes=src_nodes, det_nodes=det_nodes,
                src_ij=src_ij, det_ij=det_ij, tol=rhs_tolerances(wl),
                robin_A=wl.robin_A, k_u=wl.k_u)


def heldout_params(wl: Workload, count=1, seed_offset=1000):
    """Parameter points not used to build the basis (same jitter law)."""
    rng = np.random.default_rng(wl.seed)
    p0 = seed_params(wl, rng)
    rng2 = np.random.default_rng(wl.seed + seed_offset)
    return sample_params(wl, p0, rng2, count)


def training_params(wl: Workload, count, seed_offset=5000, n_min=2, n_max=6):
    """Phantoms of the learned augmentation's training set: each draws its
    own number of anomalies (uniform in n_min..n_max) and fresh centres,
    widths and absorptions from the seed point's law (seed_params), so they
    are not jitters of the workload's phantom.  Returns a list of parameter
    vectors (lengths differ)."""
    rng = np.random.default_rng(wl.seed + seed_offset)
    out = []
    for _ in range(count):
        na = int(rng.integers(n_min, n_max + 1))
        out.append(seed_params(replace(wl, n_anom=na), rng))
    return out
