"""ctypes binding of librcg (include/rcg.h): argument marshalling only.

Every computation happens inside the CUDA library; this module converts
numpy arrays / torch device tensors to pointers and raises on error codes.
Importing it fails loudly when the compiled library is missing: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "librcg.so")

RCG_OK = 0
RCG_ERR_INVALID = -1
RCG_ERR_CUDA = -2
RCG_ERR_OOM = -3
RCG_ERR_NOT_SPD = -4
RCG_ERR_NOT_CONVERGED = -5
RCG_ERR_BREAKDOWN = -6
RCG_ERR_TIMEOUT = -7
RCG_ERR_RANK_CAP = -8
RCG_FP64, RCG_MIXED = 0, 1
RCG_SEQUENTIAL, RCG_WAVE = 0, 1
RCG_GALERKIN, RCG_MR = 0, 1
RCG_CG, RCG_MINRES = 0, 1
RCG_INNER_OUTER, RCG_PER_RHS = 0, 1
RCG_D_FIXED, RCG_D_TRACKS_MU = 0, 1
RCG_LEARN_DEFLATE, RCG_LEARN_START = 0, 1

EXPORTED = [
    "rcg_options_default", "rcg_create", "rcg_destroy", "rcg_last_error", "rcg_strerror",
    "rcg_set_diffusion", "rcg_set_sources_detectors", "rcg_set_tolerances", "rcg_set_sample",
    "rcg_set_sample_device", "rcg_apply", "rcg_seed", "rcg_reset_to_seed", "rcg_solve_all",
    "rcg_basis_rank", "rcg_basis_get", "rcg_solution_get", "rcg_rom_eval", "rcg_rom_eval_device",
    "rcg_rom_eval_batch", "rcg_basis_compress",
    "rcg_phase_ms", "rcg_launch_count", "rcg_profile_enable", "rcg_profile_get", "rcg_apply_noalloc",
    "rcg_gemm_tn_f32", "rcg_learn_nparams", "rcg_learn_geometry", "rcg_learn_set_weights",
    "rcg_learn_get_weights", "rcg_learn_record", "rcg_learn_pairs", "rcg_learn_train", "rcg_learn_forward",
    "rcg_learn_gradient", "rcg_learn_predict", "rcg_full_eval", "rcg_save", "rcg_load", "rcg_gemm_nn_f32", "rcg_rom_eval_batch_chunk",
    "rcg_apply_f32", "rcg_stencil_variant_name", "rcg_stencil_variant_ok", "rcg_tuning_report",
    "rcg_seed_copy",
]
RCG_NOALLOC_MAX_COLS = 1024
RCG_MAX_PRIVATE = 8
RCG_STENCIL_VARIANTS = 19
RCG_COMPRESS_MAX_COLS = 4096


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("N", C.c_int), ("robin_A", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("order", C.c_int), ("wave_samples", C.c_int),
                ("tau_rank", C.c_double), ("k_u", C.c_int), ("k_cap", C.c_int), ("r_max", C.c_int),
                ("max_samples", C.c_int), ("maxit", C.c_int), ("inner_eta", C.c_double),
                ("check_refine", C.c_int), ("keep_solutions", C.c_int), ("seed_degree", C.c_int),
                ("spin_budget", C.c_longlong), ("learned", C.c_int), ("wave_rhs", C.c_int),
                ("check", C.c_int), ("inner", C.c_int), ("recycle", C.c_int),
                ("d_model", C.c_int), ("mu_s_prime", C.c_double), ("learned_mode", C.c_int)]


class Stat(C.Structure):
    _fields_ = [("sample", C.c_int), ("rhs", C.c_int), ("iters", C.c_int), ("restarts", C.c_int),
                ("appended", C.c_int), ("status", C.c_int), ("relres0", C.c_double),
                ("relres", C.c_double), ("ratio", C.c_double), ("augmented", C.c_int)]


class KProf(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("ms", C.c_double), ("lane_units", C.c_double),
                ("defl_cols", C.c_double)]


class RcgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"librcg error {code}: {msg}")
        self.code = code


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"librcg not built ({path} missing): run __graft_entry__.build()")
    lib = C.CDLL(path)
    P, I, D, LL = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    sig = {
        "rcg_options_default": (None, [C.POINTER(Options)]),
        "rcg_create": (I, [C.POINTER(P), C.POINTER(Grid), C.POINTER(Options), P]),
        "rcg_destroy": (None, [P]),
        "rcg_last_error": (C.c_char_p, [P]),
        "rcg_strerror": (C.c_char_p, [I]),
        "rcg_set_diffusion": (I, [P, P]),
        "rcg_set_sources_detectors": (I, [P, I, P, P, I, P, P]),
        "rcg_set_tolerances": (I, [P, P]),
        "rcg_set_sample": (I, [P, I, P]),
        "rcg_set_sample_device": (I, [P, I, P]),
        "rcg_apply": (I, [P, I, I, P, P, I]),
        "rcg_apply_noalloc": (I, [P, I, I, P, P, I]),
        "rcg_seed": (I, [P, I, P, P]),
        "rcg_reset_to_seed": (I, [P]),
        "rcg_solve_all": (I, [P, I, I, P]),
        "rcg_basis_rank": (I, [P, C.POINTER(I)]),
        "rcg_basis_get": (I, [P, P]),
        "rcg_solution_get": (I, [P, I, P]),
        "rcg_rom_eval": (I, [P, P, I, P, P, P]),
        "rcg_rom_eval_device": (I, [P, P, I, P, P, P]),
        "rcg_rom_eval_batch": (I, [P, I, P, I, P, P, P]),
        "rcg_basis_compress": (I, [P, I, C.c_double, P, I, C.POINTER(I)]),
        "rcg_phase_ms": (D, [P, C.c_char_p]),
        "rcg_launch_count": (LL, [P]),
        "rcg_profile_enable": (I, [P, I]),
        "rcg_profile_get": (I, [P, I, C.POINTER(KProf)]),
        "rcg_gemm_tn_f32": (I, [P, LL, I, P, LL, I, LL, P, P, I, I, I, P]),
        "rcg_learn_nparams": (I, []),
        "rcg_learn_geometry": (I, [P, P]),
        "rcg_learn_set_weights": (I, [P, P, I]),
        "rcg_learn_get_weights": (I, [P, P, I]),
        "rcg_learn_record": (I, [P, I]),
        "rcg_learn_pairs": (I, [P, C.POINTER(I)]),
        "rcg_learn_train": (I, [P, I, I, D, C.c_ulonglong, C.POINTER(D)]),
        "rcg_learn_forward": (I, [P, P, I, P]),
        "rcg_learn_gradient": (I, [P, P, P, I, P, C.POINTER(D)]),
        "rcg_learn_predict": (I, [P, I, P, P, P]),
        "rcg_full_eval": (I, [P, I, I, P, P, P]),
        "rcg_save": (I, [P, C.c_char_p]),
        "rcg_load": (I, [P, C.c_char_p]),
        "rcg_gemm_nn_f32": (I, [P, LL, I, P, I, I, LL, P, LL, D, D, I, P]),
        "rcg_rom_eval_batch_chunk": (I, [LL, I, I, I, I]),
        "rcg_apply_f32": (I, [P, I, I, P, P, I, P]),
        "rcg_stencil_variant_name": (C.c_char_p, [I]),
        "rcg_stencil_variant_ok": (I, [P, I]),
        "rcg_tuning_report": (I, [P, I]),
        "rcg_seed_copy": (I, [P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def _ptr(a):
    """Pointer of a C-contiguous numpy array or a CUDA torch tensor (or None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"] or a.flags["F_CONTIGUOUS"]
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(type(a))


def gemm_tn_f32(A, B, engine=1, symmetric=False, stream=None, w=None):
    """C = A^T diag(w) B (float64, ka x kb) for float32 CUDA tensors A (n x ka)
    and B (n x kb) stored column-major, i.e. passed as (ka, n) / (kb, n)
    row-major views (`A_cols[i]` = column i); w: float64 CUDA tensor (n) or
    None; see rcg_gemm_tn_f32."""
    import torch
    ka, n = A.shape
    kb, nb = B.shape
    assert n == nb and A.dtype == torch.float32 and B.dtype == torch.float32
    assert A.stride(1) == 1 and B.stride(1) == 1
    Cm = torch.empty((kb, ka), dtype=torch.float64, device=A.device)
    st = stream if stream is not None else torch.cuda.current_stream(A.device).cuda_stream
    if w is not None:
        assert w.dtype == torch.float64 and w.numel() >= n and w.is_contiguous()
    rc = lib().rcg_gemm_tn_f32(A.data_ptr(), A.stride(0), ka, B.data_ptr(), B.stride(0), kb, n,
                               None if w is None else w.data_ptr(), Cm.data_ptr(), ka, engine,
                               1 if symmetric else 0, st)
    if rc != 0:
        raise RcgError(rc, lib().rcg_strerror(rc).decode())
    return Cm.t()


def gemm_nn_f32(V, Cmat, Out, alpha=1.0, beta=0.0, engine=1, stream=None):
    """Out = alpha V C + beta Out in place.  V: float32 CUDA tensor (k, n) holding
    the k columns of length n; Cmat: float64 CUDA tensor (m, k) holding the m
    columns of C; Out: float32 CUDA tensor (m, n) holding the m columns of Out."""
    import torch
    k, n = V.shape
    m, k2 = Cmat.shape
    assert k == k2 and Out.shape[0] == m and Out.shape[1] == n
    assert V.dtype == torch.float32 and Cmat.dtype == torch.float64 and Out.dtype == torch.float32
    assert V.stride(1) == 1 and Cmat.stride(1) == 1 and Out.stride(1) == 1
    st = stream if stream is not None else torch.cuda.current_stream(V.device).cuda_stream
    rc = lib().rcg_gemm_nn_f32(V.data_ptr(), V.stride(0), k, Cmat.data_ptr(), Cmat.stride(0), m, n,
                               Out.data_ptr(), Out.stride(0), alpha, beta, engine, st)
    if rc != 0:
        raise RcgError(rc, lib().rcg_strerror(rc).decode())
    return Out


def stencil_variant_name(v):
    name = lib().rcg_stencil_variant_name(v)
    return None if name is None else name.decode()


def tuning_report():
    """The stencil autotuner's record (one line per tuned grid and lane class)."""
    n = lib().rcg_tuning_report(None, 0)
    buf = C.create_string_buffer(max(n, 0) + 1)
    lib().rcg_tuning_report(buf, len(buf))
    return buf.value.decode()


def default_options(**kw):
    o = Options()
    lib().rcg_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def stats_to_dicts(arr):
    return [dict(sample=s.sample, rhs=s.rhs, iters=s.iters, restarts=s.restarts, appended=s.appended,
                 status=s.status, relres0=s.relres0, relres=s.relres, ratio=s.ratio, augmented=s.augmented)
            for s in arr]


class Context:
    """One librcg context (rcg_ctx) with the same entry points as the C ABI."""

    def __init__(self, dim, N, robin_A=1.0, stream=None, **opts):
        self.L = lib()
        self.opts = default_options(**opts)
        g = Grid(dim, N, robin_A)
        h = C.c_void_p()
        s = None if stream is None else C.c_void_p(int(stream))
        self._check(self.L.rcg_create(C.byref(h), C.byref(g), C.byref(self.opts), s), None)
        self.h = h
        self.dim, self.N = dim, N
        self.n = N ** dim
        self.nsrc = self.ndet = self.nrhs = 0

    def _check(self, rc, h="self"):
        if rc != RCG_OK and rc != RCG_ERR_NOT_CONVERGED:
            msg = self.L.rcg_strerror(rc).decode()
            if h is not None:
                msg += ": " + self.L.rcg_last_error(self.h).decode()
            raise RcgError(rc, msg)
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.L.rcg_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- inputs
    def set_diffusion(self, D):
        D = np.ascontiguousarray(D, dtype=np.float64)
        return self._check(self.L.rcg_set_diffusion(self.h, _ptr(D)))

    def set_sources_detectors(self, src_ij, det_ij, src_w=None, det_w=None):
        s = np.ascontiguousarray(src_ij, dtype=np.int32).reshape(-1, 2)
        d = np.ascontiguousarray(det_ij, dtype=np.int32).reshape(-1, 2)
        sw = None if src_w is None else np.ascontiguousarray(src_w, dtype=np.float64)
        dw = None if det_w is None else np.ascontiguousarray(det_w, dtype=np.float64)
        self.nsrc, self.ndet = len(s), len(d)
        self.nrhs = self.nsrc + self.ndet
        return self._check(self.L.rcg_set_sources_detectors(self.h, len(s), _ptr(s), _ptr(sw),
                                                            len(d), _ptr(d), _ptr(dw)))

    def set_tolerances(self, tol):
        t = np.ascontiguousarray(tol, dtype=np.float64)
        return self._check(self.L.rcg_set_tolerances(self.h, _ptr(t)))

    def set_sample(self, s, mu):
        if hasattr(mu, "data_ptr"):
            return self._check(self.L.rcg_set_sample_device(self.h, s, _ptr(mu)))
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        return self._check(self.L.rcg_set_sample(self.h, s, _ptr(mu)))

    def _device_cols(self, x_dev, y_dev, ncols, prec):
        """x and y must be contiguous CUDA tensors of the precision's dtype
        (float64 for RCG_FP64, float32 for RCG_MIXED) holding ncols columns of
        n values: anything else would hand the kernel a host or out-of-bounds
        address."""
        import torch
        want = torch.float64 if prec == RCG_FP64 else torch.float32
        for name, t in (("x", x_dev), ("y", y_dev)):
            if not isinstance(t, torch.Tensor) or not t.is_cuda:
                raise ValueError(f"{name} must be a CUDA tensor")
            if t.dtype != want or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous {want} tensor for prec {prec}")
            if ncols < 0 or t.numel() < ncols * self.n:
                raise ValueError(f"{name} holds {t.numel()} values, fewer than ncols * n = {ncols * self.n}")

    def apply(self, s, x_dev, y_dev, ncols, prec=RCG_FP64):
        self._device_cols(x_dev, y_dev, ncols, prec)
        return self._check(self.L.rcg_apply(self.h, s, prec, _ptr(x_dev), _ptr(y_dev), ncols))

    def apply_noalloc(self, s, x_dev, y_dev, ncols, prec=RCG_FP64):
        """rcg_apply without device allocation (tables in a static device array)."""
        if 0 <= ncols <= RCG_NOALLOC_MAX_COLS:
            self._device_cols(x_dev, y_dev, ncols, prec)
        return self._check(self.L.rcg_apply_noalloc(self.h, s, prec, _ptr(x_dev), _ptr(y_dev), ncols))

    def apply_f32(self, s, x_dev, y_dev, ncols, variant=-1, dots_dev=None):
        """y = A~_s x with the inner iteration's float32 stencil kernel
        `variant` (-1: the autotuned choice); dots_dev[j] += x_j^T y_j."""
        self._device_cols(x_dev, y_dev, ncols, RCG_MIXED)
        if dots_dev is not None:
            import torch
            if not (isinstance(dots_dev, torch.Tensor) and dots_dev.is_cuda and dots_dev.dtype == torch.float64
                    and dots_dev.numel() >= ncols):
                raise ValueError("dots must be a CUDA float64 tensor of ncols values")
        return self._check(self.L.rcg_apply_f32(self.h, s, variant, _ptr(x_dev), _ptr(y_dev), ncols, _ptr(dots_dev)))

    def stencil_variant_ok(self, v):
        return bool(self.L.rcg_stencil_variant_ok(self.h, v))

    # ---- method
    def seed(self, s0, U0=None):
        st = (Stat * self.nrhs)()
        U = None if U0 is None else np.asfortranarray(U0, dtype=np.float64)
        self._check(self.L.rcg_seed(self.h, s0, _ptr(U), st))
        return stats_to_dicts(st)

    def seed_copy(self, src):
        """rcg_seed_copy: take the seed state of Context `src`."""
        return self._check(self.L.rcg_seed_copy(self.h, src.h))

    def reset_to_seed(self):
        return self._check(self.L.rcg_reset_to_seed(self.h))

    def solve_all(self, s_first, s_count, want_stats=True):
        st = (Stat * (self.nrhs * s_count))() if want_stats else None
        rc = self._check(self.L.rcg_solve_all(self.h, s_first, s_count, st))
        return (stats_to_dicts(st) if want_stats else None), rc

    def rank(self):
        r = C.c_int()
        self._check(self.L.rcg_basis_rank(self.h, C.byref(r)))
        return r.value

    def basis(self):
        r = self.rank()
        V = np.zeros((self.n, r), dtype=np.float64, order="F")
        self._check(self.L.rcg_basis_get(self.h, _ptr(V)))
        return V

    def solutions(self, s):
        X = np.zeros((self.n, self.nrhs), dtype=np.float64, order="F")
        self._check(self.L.rcg_solution_get(self.h, s, _ptr(X)))
        return X

    def rom_eval(self, mu, dmu=None):
        """Psi_r (ndet, nsrc) and J_r (nparam, ndet, nsrc) or None."""
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        Psi = np.zeros((self.ndet, self.nsrc), dtype=np.float64, order="F")
        if dmu is None:
            self._check(self.L.rcg_rom_eval(self.h, _ptr(mu), 0, None, _ptr(Psi), None))
            return Psi, None
        dmu = np.ascontiguousarray(dmu, dtype=np.float64)     # (nparam, n) C order = n x nparam col-major
        k = dmu.shape[0]
        J = np.zeros((k, self.nsrc, self.ndet), dtype=np.float64)   # C order = J[d + ndet*(s + nsrc*k)]
        self._check(self.L.rcg_rom_eval(self.h, _ptr(mu), k, _ptr(dmu), _ptr(Psi), _ptr(J)))
        return Psi, np.transpose(J, (0, 2, 1))

    def save(self, path):
        return self._check(self.L.rcg_save(self.h, os.fsencode(path)))

    def load(self, path):
        return self._check(self.L.rcg_load(self.h, os.fsencode(path)))

    def full_eval(self, s, dmu=None):
        """Psi (ndet x nsrc) and J (nparam x ndet x nsrc) from the kept solutions of sample s."""
        Psi = np.zeros((self.ndet, self.nsrc), dtype=np.float64, order="F")
        J = None
        k = 0
        if dmu is not None:
            dmu = np.ascontiguousarray(dmu, dtype=np.float64)      # (nparam, n) -> n x nparam column-major
            k = dmu.shape[0]
            J = np.zeros((k, self.nsrc, self.ndet), dtype=np.float64)
        self._check(self.L.rcg_full_eval(self.h, s, k, _ptr(dmu), _ptr(Psi), _ptr(J)))
        return Psi, (None if J is None else np.transpose(J, (0, 2, 1)))

    def rom_eval_device(self, mu_dev, dmu_dev, Psi_dev, J_dev, nparam):
        return self._check(self.L.rcg_rom_eval_device(self.h, _ptr(mu_dev), nparam, _ptr(dmu_dev),
                                                      _ptr(Psi_dev), _ptr(J_dev)))

    def basis_compress(self, r_max=0, tau=1e-8, sigma_len=1 << 16):
        """rcg_basis_compress: returns (new rank, singular values of the snapshot matrix)."""
        sig = np.zeros(sigma_len, dtype=np.float64)
        m = C.c_int(0)
        self._check(self.L.rcg_basis_compress(self.h, int(r_max), float(tau), _ptr(sig), sigma_len, C.byref(m)))
        return self.rank(), sig[: min(m.value, sigma_len)].copy()

    def rom_eval_batch_device(self, nq, mu_dev, dmu_dev, Psi_dev, J_dev, nparam):
        """rcg_rom_eval_batch on device arrays (see rcg.h for the layouts)."""
        return self._check(self.L.rcg_rom_eval_batch(self.h, nq, _ptr(mu_dev), nparam, _ptr(dmu_dev),
                                                     _ptr(Psi_dev), _ptr(J_dev)))

    def rom_eval_batch(self, mus, dmus=None):
        """Psi (nq, ndet, nsrc) and J (nq, nparam, ndet, nsrc) or None at the
        rows of mus (nq, n), through device copies made with torch."""
        import torch
        mus = np.ascontiguousarray(mus, dtype=np.float64)
        nq = mus.shape[0]
        dev = torch.device("cuda", torch.cuda.current_device())
        mu_d = torch.from_numpy(mus).to(dev)
        Psi_d = torch.empty((nq, self.nsrc, self.ndet), dtype=torch.float64, device=dev)
        dmu_d = J_d = None
        k = 0
        if dmus is not None:
            dmus = np.ascontiguousarray(dmus, dtype=np.float64)
            k = dmus.shape[1]
            dmu_d = torch.from_numpy(dmus).to(dev)
            J_d = torch.empty((nq, k, self.nsrc, self.ndet), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        self.rom_eval_batch_device(nq, mu_d, dmu_d, Psi_d, J_d, k)
        Psi = Psi_d.cpu().numpy().transpose(0, 2, 1)
        J = None if J_d is None else J_d.cpu().numpy().transpose(0, 1, 3, 2)
        return Psi, J

    def phase_ms(self, name):
        return self.L.rcg_phase_ms(self.h, name.encode())

    def launch_count(self):
        return self.L.rcg_launch_count(self.h)

    def profile(self, on=True):
        return self._check(self.L.rcg_profile_enable(self.h, 1 if on else 0))

    def profile_get(self, kernel):
        k = KProf()
        self._check(self.L.rcg_profile_get(self.h, kernel, C.byref(k)))
        return dict(launches=k.launches, ms=k.ms, lane_units=k.lane_units, defl_cols=k.defl_cols)

    # ---- learned augmentation (rcg_learn_*)
    def learn_geometry(self):
        d = np.zeros(4, dtype=np.int32)
        self._check(self.L.rcg_learn_geometry(self.h, _ptr(d)))
        return tuple(int(v) for v in d)          # Gx, Gy, Gz, f

    def learn_set_weights(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        return self._check(self.L.rcg_learn_set_weights(self.h, _ptr(t), t.size))

    def learn_get_weights(self):
        t = np.zeros(self.L.rcg_learn_nparams(), dtype=np.float32)
        self._check(self.L.rcg_learn_get_weights(self.h, _ptr(t), t.size))
        return t

    def learn_record(self, on=True):
        return self._check(self.L.rcg_learn_record(self.h, 1 if on else 0))

    def learn_pairs(self):
        v = C.c_int()
        self._check(self.L.rcg_learn_pairs(self.h, C.byref(v)))
        return v.value

    def learn_train(self, epochs, batch=16, lr=1e-3, seed=0):
        loss = C.c_double()
        self._check(self.L.rcg_learn_train(self.h, epochs, batch, lr, seed, C.byref(loss)))
        return loss.value

    def learn_forward(self, inp):
        x = np.ascontiguousarray(inp, dtype=np.float32)
        B = x.shape[0]
        out = np.zeros((B,) + x.shape[2:], dtype=np.float32)
        self._check(self.L.rcg_learn_forward(self.h, _ptr(x), B, _ptr(out)))
        return out

    def learn_gradient(self, inp, tg):
        x = np.ascontiguousarray(inp, dtype=np.float32)
        t = np.ascontiguousarray(tg, dtype=np.float32)
        g = np.zeros(self.L.rcg_learn_nparams(), dtype=np.float32)
        loss = C.c_double()
        self._check(self.L.rcg_learn_gradient(self.h, _ptr(x), _ptr(t), x.shape[0], _ptr(g), C.byref(loss)))
        return loss.value, g

    def learn_predict(self, s, r0):
        Gx, Gy, Gz, _ = self.learn_geometry()
        r = np.ascontiguousarray(r0, dtype=np.float32)
        feat = np.zeros((2, Gz, Gy, Gx), dtype=np.float32)
        xhat = np.zeros(self.n, dtype=np.float32)
        self._check(self.L.rcg_learn_predict(self.h, s, _ptr(r), _ptr(feat), _ptr(xhat)))
        return feat, xhat
