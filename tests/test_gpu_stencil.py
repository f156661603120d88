"""Every float32 stencil kernel of the inner CG iteration (rcg_apply_f32,
variants 0..RCG_STENCIL_VARIANTS-1: the row kernel, the plane ring and the
z-marching tiles with 1, 2 or 4 lanes per CTA, in both grid orders, and two
with registers for three CTAs per SM, and the TMA plane-ring kernels on the
grids whose Nx is a multiple of 64) against the oracle's operator
A~_s (the numerically formed Schur complement of the full finite-difference
system, Sec. 3) on grids with one and several x-tiles, a ragged y-tile
(80 rows in tiles of 64) and a z-chunk boundary, plus the fused p^T q.

Tolerance: |y - y_ref| <= 2e-6 ||A~||_inf |x|_inf (float32 products of seven
terms), p^T q within 1e-5 relative of the float64 value."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import operator as op
from synthetic.phantom import WORKLOADS, make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rcg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1602_00138_gb300 import rcg as r
    return r


@pytest.mark.parametrize("N", [16, 32, 48, 64, 80, 128])
def test_every_stencil_variant_matches_the_oracle_operator(rcg, N):
    import torch
    wl = replace(WORKLOADS["t3d_16"], name=f"t3d_{N}", N=N)
    inp = make_workload(wl, with_dmu=False)
    A, _, _ = op.assemble(inp, 1)
    rng = np.random.default_rng(N)
    ncols = 5
    X = rng.standard_normal((ncols, wl.n)).astype(np.float32)
    Y_ref = (A @ X.astype(np.float64).T).T
    scale = abs(A).sum(axis=1).max() * np.abs(X).max()
    d_ref = np.einsum("ij,ij->i", X.astype(np.float64), Y_ref)
    ran = []
    with rcg.Context(wl.dim, wl.N, wl.robin_A) as ctx:
        ctx.set_diffusion(inp["D"])
        ctx.set_sample(1, inp["mu"][1])
        x = torch.tensor(X, device="cuda")
        for v in list(range(rcg.RCG_STENCIL_VARIANTS)) + [-1]:
            if v >= 0 and not ctx.stencil_variant_ok(v):
                with pytest.raises(rcg.RcgError):
                    ctx.apply_f32(1, x, torch.empty_like(x), ncols, variant=v)
                continue
            y = torch.full_like(x, float("nan"))
            dots = torch.zeros(ncols, dtype=torch.float64, device="cuda")
            ctx.apply_f32(1, x, y, ncols, variant=v, dots_dev=dots)
            torch.cuda.synchronize()
            err = np.abs(y.double().cpu().numpy() - Y_ref).max() / scale
            assert err <= 2e-6, (v, rcg.stencil_variant_name(v), err)
            dd = dots.cpu().numpy()
            assert np.allclose(dd, d_ref, rtol=1e-5, atol=0), (v, dd, d_ref)
            ran.append(v)
    # the z-marching tiles run wherever Nx / 4 is a multiple of 4, the TMA tiles where Nx % 64 == 0
    if (N // 4) % 4 == 0:
        assert any(v >= 2 for v in ran)
    if N % 64 == 0:
        assert {16, 17, 18} <= set(ran)
    assert "stencil" in rcg.tuning_report()


def test_tile_first_grid_order_with_many_lanes(rcg):
    """37 columns (19 lane groups of two, a ragged last group): the tile-first
    grid order that more than 16 groups take, every z-marching variant, against
    the oracle's operator."""
    import torch
    wl = replace(WORKLOADS["t3d_16"], name="t3d_32c", N=32)
    inp = make_workload(wl, with_dmu=False)
    A, _, _ = op.assemble(inp, 1)
    rng = np.random.default_rng(37)
    ncols = 37
    X = rng.standard_normal((ncols, wl.n)).astype(np.float32)
    Y_ref = (A @ X.astype(np.float64).T).T
    scale = abs(A).sum(axis=1).max() * np.abs(X).max()
    with rcg.Context(wl.dim, wl.N, wl.robin_A) as ctx:
        ctx.set_diffusion(inp["D"])
        ctx.set_sample(1, inp["mu"][1])
        x = torch.tensor(X, device="cuda")
        for v in range(2, rcg.RCG_STENCIL_VARIANTS):
            if not ctx.stencil_variant_ok(v):
                continue
            y = torch.full_like(x, float("nan"))
            ctx.apply_f32(1, x, y, ncols, variant=v)
            torch.cuda.synchronize()
            err = np.abs(y.double().cpu().numpy() - Y_ref).max() / scale
            assert err <= 2e-6, (v, rcg.stencil_variant_name(v), err)
