"""The C-ABI library builds, loads and exports every entry point declared in
include/rcg.h (no GPU needed: nothing here launches device work)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "rcg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rcg_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1602_00138_gb300 import rcg
    return rcg.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1602_00138_gb300 import rcg
    assert sorted(rcg.EXPORTED) == names


def test_binding_argument_counts_match_the_header(lib):
    """Every binding signature takes as many arguments as the header's
    prototype declares (a mismatch would pass garbage through ctypes)."""
    txt = open(os.path.join(ROOT, "include", "rcg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = dict(re.findall(r"\b(rcg_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", txt, flags=re.S))
    checked = 0
    for name in _declared():
        if name not in protos:
            continue
        params = protos[name].strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(getattr(lib, name).argtypes) == n, (name, params)
        checked += 1
    assert checked >= 40


def test_host_only_entry_points(lib):
    from paper_1602_00138_gb300 import rcg
    o = rcg.default_options()
    assert o.precision == rcg.RCG_FP64 and o.k_u == 10 and o.tau_rank == 1e-12
    assert lib.rcg_strerror(rcg.RCG_ERR_RANK_CAP) == b"basis rank cap reached"
    assert lib.rcg_strerror(0) == b"ok"
    # invalid grids are rejected before any device work
    import ctypes as C
    h = C.c_void_p()
    bad = rcg.Grid(4, 10, 1.0)
    assert lib.rcg_create(C.byref(h), C.byref(bad), None, None) == rcg.RCG_ERR_INVALID
    bad = rcg.Grid(3, 10, -1.0)
    assert lib.rcg_create(C.byref(h), C.byref(bad), None, None) == rcg.RCG_ERR_INVALID
    assert lib.rcg_launch_count(None) == -1


def test_header_constants_match_the_binding():
    """Every RCG_* integer constant of include/rcg.h that the binding mirrors has the same value."""
    from paper_1602_00138_gb300 import rcg
    txt = open(os.path.join(ROOT, "include", "rcg.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+(RCG_[A-Z_0-9]+)\s+(-?\d+)", txt)}
    mirrored = [k for k in defs if hasattr(rcg, k)]
    assert {"RCG_OK", "RCG_ERR_INVALID", "RCG_MIXED", "RCG_WAVE", "RCG_NOALLOC_MAX_COLS",
            "RCG_COMPRESS_MAX_COLS", "RCG_MAX_PRIVATE"} <= set(mirrored)
    for k in mirrored:
        assert getattr(rcg, k) == defs[k], k


def test_rom_batch_chunk_bounds_the_workspace(lib):
    """rcg_rom_eval_batch splits its points so that the workspace stays within
    RCG_ROM_BATCH_WORKSPACE (4 GiB): at the 192^3 configuration (basis of
    2048 columns, 128 + 128 right-hand sides, 40 parameters) a point needs
    about 2 GB (40 Grams of 2048^2 float64 and their float32 partial sums), so
    two points go together where 256 needed ~515 GB; small bases take the
    full 256-point chunks.  Host arithmetic only (nothing allocated)."""
    n = 192 ** 3
    assert lib.rcg_rom_eval_batch_chunk(n, 2048, 128, 128, 40) == 2
    assert lib.rcg_rom_eval_batch_chunk(n, 2048, 128, 128, 0) >= 1
    assert lib.rcg_rom_eval_batch_chunk(64 ** 3, 120, 32, 32, 20) == 256
    assert lib.rcg_rom_eval_batch_chunk(-1, 10, 1, 1, 1) == -1
    # the bound itself: per point ~ nparam r^2 (8 B Gram + 4 B partial sums) at r = 512
    k = lib.rcg_rom_eval_batch_chunk(128 ** 3, 512, 64, 64, 20)
    per = 20 * 512 * 512 * 12 + 8 * 128 ** 3
    assert (k - 1) * per <= 4 * 2 ** 30 and k >= 1


def test_binding_refuses_host_or_short_operands(lib):
    """apply / apply_noalloc check their operands before the library sees a
    pointer: numpy arrays, CPU tensors and wrong dtypes are refused (no GPU
    needed: the check runs before any call)."""
    import numpy as np
    import torch
    from paper_1602_00138_gb300 import rcg
    ctx = rcg.Context.__new__(rcg.Context)
    ctx.n = 10
    with pytest.raises(ValueError):
        ctx._device_cols(np.zeros(20), np.zeros(20), 2, rcg.RCG_FP64)
    with pytest.raises(ValueError):
        ctx._device_cols(torch.zeros(20, dtype=torch.float64), torch.zeros(20, dtype=torch.float64), 2,
                         rcg.RCG_FP64)
