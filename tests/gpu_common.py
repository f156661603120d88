"""Shared helpers of the GPU parity tests: run a workload through the C ABI
(via the ctypes binding) and through the FP64 CPU oracle, on the same seeded
synthetic inputs."""
import functools

import numpy as np

from oracle import basis as obasis, eigen, operator as op, rom
from synthetic.phantom import make_workload


@functools.lru_cache(maxsize=None)
def workload(name):
    return make_workload(name)


@functools.lru_cache(maxsize=None)
def oracle_seed_inputs(name):
    inp = workload(name)
    A0, Bt, Ct = op.assemble(inp, 0)
    _, U0 = eigen.smallest_eigenpairs(A0, inp["wl"].k_u)
    As = {i: op.assemble(inp, i)[0] for i in range(inp["wl"].K + 1)}
    return U0, As, Bt, Ct


@functools.lru_cache(maxsize=None)
def oracle_run(name, order, tau):
    inp = workload(name)
    wl = inp["wl"]
    U0, As, Bt, Ct = oracle_seed_inputs(name)
    B = np.hstack([Bt, Ct])
    st = obasis.seed(As[0], B, U0, inp["tol"], tau=tau)
    seed_stats = list(st.stats)
    out = obasis.solve_all(st, lambda i: As[i], range(1, wl.K + 1), B, inp["tol"], order=order, tau=tau)
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
