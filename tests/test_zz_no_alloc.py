"""rcg_apply_noalloc against rcg_apply through the C ABI.

rcg_apply_noalloc serves callers that cannot allocate device memory during
the call (device memory owned by another allocator, or no cudaMalloc /
cudaFree allowed on a repeated call): it keeps its per-column tables in a
static device array of the library instead of allocating them.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process and after the others.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["t3d_21", "t2d_37"])
def test_noalloc_apply_matches_apply_on_two_calls(name):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1602_00138_gb300 import rcg
    from synthetic.phantom import make_workload
    inp = make_workload(name)
    wl = inp["wl"]
    rng = np.random.default_rng(11)
    with rcg.Context(wl.dim, wl.N, wl.robin_A) as ctx:
        ctx.set_diffusion(inp["D"])
        ctx.set_sample(1, inp["mu"][1])
        for call, ncols in enumerate((7, 3)):                 # two calls in a row
            for prec, dt, tol in ((rcg.RCG_FP64, torch.float64, 1e-14), (rcg.RCG_MIXED, torch.float32, 1e-6)):
                x = torch.tensor(rng.standard_normal((ncols, wl.n)), dtype=dt, device="cuda")
                y_ref = torch.empty_like(x)
                y = torch.full_like(x, float("nan"))
                ctx.apply(1, x, y_ref, ncols, prec)
                ctx.apply_noalloc(1, x, y, ncols, prec)
                torch.cuda.synchronize()
                err = (y - y_ref).abs().max().item() / y_ref.abs().max().item()
                assert err <= tol, (call, prec, err)
        # sizes beyond the static array are rejected with an error, not run
        big = rcg.RCG_NOALLOC_MAX_COLS + 1
        with pytest.raises(rcg.RcgError) as e:
            ctx.apply_noalloc(1, x, y, big, rcg.RCG_MIXED)
        assert e.value.code == rcg.RCG_ERR_INVALID
