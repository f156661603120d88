"""Shared helpers of the GPU parity tests: run a workload through the C ABI
(via the ctypes binding) and through the FP64 CPU oracle, on the same seeded
synthetic inputs."""
import functools

import numpy as np

from oracle import basis as obasis, eigen, operator as op, rom
from synthetic.phantom import make_workload


_SEED_LAMBDA = {}


@functools.lru_cache(maxsize=None)
def workload(name):
    return make_workload(name)


@functools.lru_cache(maxsize=None)
def oracle_seed_inputs(name):
    inp = workload(name)
    A0, Bt, Ct = op.assemble(inp, 0)
    w, U0 = eigen.smallest_eigenpairs(A0, inp["wl"].k_u)
    _SEED_LAMBDA[name] = float(w[0])
    As = {i: op.assemble(inp, i)[0] for i in range(inp["wl"].K + 1)}
    return U0, As, Bt, Ct


def effective_cap(k_u, k_cap):
    """The library's bound on the columns of U_j: k_cap, but at most k_u +
    RCG_MAX_PRIVATE (8) private columns (include/rcg.h, rcg_options.k_cap)."""
    return min(k_cap, k_u + 8)


@functools.lru_cache(maxsize=None)
def oracle_run(name, order, tau, k_cap=256, wave_samples=0, wave_rhs=0):
    inp = workload(name)
    wl = inp["wl"]
    U0, As, Bt, Ct = oracle_seed_inputs(name)
    B = np.hstack([Bt, Ct])
    st = obasis.seed(As[0], B, U0, inp["tol"], tau=tau, k_cap=effective_cap(wl.k_u, k_cap))
    seed_stats = list(st.stats)
    out = obasis.solve_all(st, lambda i: As[i], range(1, wl.K + 1), B, inp["tol"], order=order, tau=tau,
                           wave_samples=wave_samples, wave_rhs=wave_rhs)
    return st, seed_stats, out


def gpu_run(name, precision, order, tau, wave_samples=0, k_cap=256, **kw):
    from paper_1602_00138_gb300 import rcg
    inp = workload(name)
    wl = inp["wl"]
    U0, _, _, _ = oracle_seed_inputs(name)
    opts = dict(k_u=wl.k_u, keep_solutions=1, wave_samples=wave_samples, k_cap=k_cap)
    opts.update(kw)
    ctx = rcg.Context(wl.dim, wl.N, wl.robin_A, precision=precision, order=order, tau_rank=tau, **opts)
    ctx.set_diffusion(inp["D"])
    ctx.set_sources_detectors(inp["src_ij"], inp["det_ij"])
    ctx.set_tolerances(inp["tol"])
    for s in range(wl.K + 1):
        ctx.set_sample(s, inp["mu"][s])
    seed_stats = ctx.seed(0, U0)
    r_seed = ctx.rank()
    stats, rc = ctx.solve_all(1, wl.K)
    return ctx, seed_stats, stats, rc, r_seed


def ambiguous(stats, tols, tau, band=10.0):
    """Decisions inside the guard band: relres0/tol or ratio/tau in [1/band, band]."""
    amb = 0
    for s in stats:
        t = tols[s["rhs"]]
        if 1.0 / band <= s["relres0"] / t <= band:
            amb += 1
        elif s["iters"] > 0 and s.get("ratio", 0) > 0 and 1.0 / band <= s["ratio"] / tau <= band:
            amb += 1
    return amb


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def jacobian_galerkin_bound(A, Bt, Ct, h, dmu, tol, tau_eff, lam_min):
    """Relative Frobenius bound on J_r - J at a sampled point (eq. newjac,
    Theorem of Sec. 3.4 with inexact solves).

    x_s = A~^-1 b~_s and z_d = A~^-1 c~_d; the reduced model's x_r = P x_s is
    the A~-orthogonal projection onto range(V).  A delivered solution x' met
    ||b - A~ x'|| <= tol ||b|| and lies in range(V) up to a dropped part of
    relative size tau_eff (the append's drop test plus the basis storage), so
        ||x - x_r||_A <= tol ||b|| / sqrt(lam_min) + sqrt(lam_max) tau_eff ||x||,
        ||x - x_r||_2 <= ||x - x_r||_A / sqrt(lam_min) =: e_x.
    J_r - J = -(e_z^T Delta_k x + z^T Delta_k e_x + e_z^T Delta_k e_x), hence
        |J_r - J|_{k,d,s} <= ||Delta_k||_2 (e_z ||x|| + ||z|| e_x + e_z e_x),
    ||Delta_k||_2 = h^2 max |dmu_k|.  First order in the solve tolerance, so
    two reduced models built from different bases that both meet tol agree
    only to twice this, not to the float64 rounding level."""
    from oracle.solvers import direct_solve
    X = direct_solve(A, Bt)
    Z = direct_solve(A, Ct)
    lam_max = abs(A).sum(axis=1).max()                 # Gershgorin bound of the SPD A~
    ns, nd = Bt.shape[1], Ct.shape[1]
    tol = np.broadcast_to(np.asarray(tol, dtype=np.float64), (ns + nd,))

    def err(x, b, t):
        eA = t * np.linalg.norm(b) / np.sqrt(lam_min) + np.sqrt(lam_max) * tau_eff * np.linalg.norm(x)
        return eA / np.sqrt(lam_min)

    ex = np.array([err(X[:, s], Bt[:, s], tol[s]) for s in range(ns)])
    ez = np.array([err(Z[:, d], Ct[:, d], tol[ns + d]) for d in range(nd)])
    nx, nz = np.linalg.norm(X, axis=0), np.linalg.norm(Z, axis=0)
    per = ez[:, None] * nx[None, :] + nz[:, None] * ex[None, :] + ez[:, None] * ex[None, :]   # (nd, ns)
    dn = h * h * np.abs(dmu).max(axis=1)                                                     # (nparam,)
    J = np.stack([-(Z.T @ ((h * h * dmu[k])[:, None] * X)) for k in range(dmu.shape[0])])
    bound = np.sqrt(np.sum(dn ** 2) * np.sum(per ** 2))
    return float(bound / np.linalg.norm(J)), J


def lambda_min_lower(name, s):
    """A lower bound on the smallest eigenvalue of A~_s by Weyl's inequality:
    A~_s = A~_0 + diag(h^2 (mu_s - mu_0)), so lambda_min(A~_s) >=
    lambda_min(A~_0) + h^2 min(mu_s - mu_0), with lambda_min(A~_0) from the
    oracle's seed eigensolver (dense LAPACK or ARPACK)."""
    inp = workload(name)
    oracle_seed_inputs(name)
    return float(_SEED_LAMBDA[name] + inp["h"] ** 2 * np.min(inp["mu"][s] - inp["mu"][0]))
