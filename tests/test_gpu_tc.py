"""GPU tests of the basis product C = A^T B (rcg_gemm_tn_f32), the
orthogonalisation product of the append (Sec. 5.3 incremental QR), on the
tensor cores (engine 1, tcgen05 3xTF32) and on CUDA cores (engine 0).

Reference: the float64 product of the same float32 inputs, computed by numpy
on the host.  The error of entry (i, j) is measured against
||a_i|| ||b_j|| (the scale of its rounding errors).  Positive data is the hard
case for accumulation (every product has the same sign); ragged n, ka, kb and
a leading dimension that is a multiple of 4 but not of 32 cover the partial
tiles, the zero-filled tails and the copy alignment.
"""
import numpy as np
import pytest

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


def _cols(rng, k, n, ld, positive):
    X = np.zeros((k, ld), dtype=np.float32)
    X[:, :n] = rng.random((k, n), dtype=np.float32) - (0.0 if positive else 0.5)
    return X


def _run(rcg, n, ka, kb, positive, engine, symmetric=False):
    import torch
    rng = np.random.default_rng(1000 * ka + kb)
    ld = (n + 63) // 64 * 64 + 4
    A = _cols(rng, ka, n, ld, positive)
    B = A if symmetric else _cols(rng, kb, n, ld, positive)
    dA = torch.from_numpy(A).cuda()
    dB = dA if symmetric else torch.from_numpy(B).cuda()
    C = rcg.gemm_tn_f32(dA[:, :n], dB[:, :n], engine=engine, symmetric=symmetric)
    C = C.cpu().numpy()
    A64, B64 = A[:, :n].astype(np.float64), B[:, :n].astype(np.float64)
    ref = A64 @ B64.T
    scale = np.outer(np.linalg.norm(A64, axis=1), np.linalg.norm(B64, axis=1))
    scale[scale == 0] = 1.0
    return float(np.max(np.abs(C - ref) / scale)) if C.size else 0.0


CASES = [(100003, 150, 70, False), (70001, 7, 300, True), (40, 5, 3, False), (262144, 130, 129, True),
         (4096, 128, 128, True)]


@pytest.mark.parametrize("n,ka,kb,positive", CASES)
def test_tensor_core_product_matches_float64(rcg, n, ka, kb, positive):
    err = _run(rcg, n, ka, kb, positive, engine=1)
    assert err <= 5e-7, err


@pytest.mark.parametrize("n,ka,kb,positive", CASES[:3])
def test_cuda_core_product_matches_float64(rcg, n, ka, kb, positive):
    err = _run(rcg, n, ka, kb, positive, engine=0)
    assert err <= 1e-7, err


@pytest.mark.parametrize("n,k", [(50001, 260), (262144, 320)])
def test_symmetric_tensor_core_product(rcg, n, k):
    err = _run(rcg, n, k, k, True, engine=1, symmetric=True)
    assert err <= 5e-7, err


def test_empty_and_invalid_arguments(rcg):
    import torch
    A = torch.zeros((4, 64), dtype=torch.float32, device="cuda")
    # n = 0: C = 0
    C = rcg.gemm_tn_f32(A[:, :0], A[:, :0], engine=1)
    assert C.shape == (4, 4) and float(C.abs().max()) == 0.0
    # leading dimension not a multiple of 4: refused on the host for the tensor cores
    B = torch.zeros((4, 63), dtype=torch.float32, device="cuda")
    with pytest.raises(rcg.RcgError) as e:
        rcg.gemm_tn_f32(B, B, engine=1)
    assert e.value.code == rcg.RCG_ERR_INVALID
    # symmetric with different operands
    with pytest.raises(rcg.RcgError):
        rcg.gemm_tn_f32(A, A.clone(), engine=1, symmetric=True)


@pytest.mark.parametrize("engine", [1, 0])
def test_weighted_product_with_finite_support(rcg, engine):
    """C = A^T diag(w) A with w zero outside a few scattered ranges (the check's
    Delta weights have finite support): the tensor cores visit only the
    32-row blocks where w does not vanish."""
    import torch
    n, k = 100003, 130
    rng = np.random.default_rng(21)
    ld = (n + 63) // 64 * 64
    A = np.zeros((k, ld), dtype=np.float32)
    A[:, :n] = rng.random((k, n), dtype=np.float32)
    w = np.zeros(ld)
    for a, b in [(5, 40), (1000, 1031), (50000, 57777), (99990, 100003)]:
        w[a:b] = rng.random(b - a) * 1e-3
    dA = torch.from_numpy(A).cuda()
    dw = torch.from_numpy(w).cuda()
    C = rcg.gemm_tn_f32(dA[:, :n], dA[:, :n], engine=engine, symmetric=(engine == 1), w=dw).cpu().numpy()
    A64 = A[:, :n].astype(np.float64)
    ref = (A64 * w[:n]) @ A64.T
    scale = np.outer(np.linalg.norm(A64 * np.sqrt(w[:n]), axis=1), np.linalg.norm(A64 * np.sqrt(w[:n]), axis=1))
    err = np.max(np.abs(C - ref) / scale)
    assert err <= (5e-7 if engine == 1 else 1e-7), err


NN_CASES = [(100003, 150, 70, False, 0.0), (70001, 7, 300, True, 1.0), (40, 33, 20, False, -1.0),
            (262144, 130, 129, True, 1.0), (4096, 128, 128, True, 0.0)]


@pytest.mark.parametrize("n,k,m,positive,beta", NN_CASES)
@pytest.mark.parametrize("engine", [1, 0])
def test_update_product_matches_float64(rcg, n, k, m, positive, beta, engine):
    """Out = alpha V C + beta Out (the append's basis updates) against float64."""
    import torch
    rng = np.random.default_rng(100 * k + m)
    ld = (n + 63) // 64 * 64 + 4
    V = _cols(rng, k, n, ld, positive)
    Cm = rng.standard_normal((m, k)) * (1.0 if not positive else 0.1)
    O = _cols(rng, m, n, ld, positive)
    dV = torch.from_numpy(V).cuda()
    dC = torch.from_numpy(Cm).cuda()
    dO = torch.from_numpy(O.copy()).cuda()
    alpha = -0.75
    rcg.gemm_nn_f32(dV[:, :n], dC, dO[:, :n], alpha=alpha, beta=beta, engine=engine)
    out = dO.cpu().numpy()[:, :n].astype(np.float64)
    V64 = V[:, :n].astype(np.float64)
    ref = alpha * (Cm.astype(np.float32).astype(np.float64) @ V64) + beta * O[:, :n].astype(np.float64)
    # rounding scale of entry (j, p): |alpha| sum_i |C_ij V_ip| + |beta O_jp|
    scale = abs(alpha) * (np.abs(Cm) @ np.abs(V64)) + abs(beta) * np.abs(O[:, :n]) + 1e-30
    err = np.max(np.abs(out - ref) / scale)
    assert err <= 4e-6, err
    # the padding beyond n is untouched
    assert np.array_equal(dO.cpu().numpy()[:, n:], O[:, n:])
