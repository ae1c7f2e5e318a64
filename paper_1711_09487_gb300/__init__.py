"""GB300-native RF-DDES interface rational filter (arXiv:1711.09487) -- Python binding.

A thin ctypes layer over the C ABI declared in ``include/rfdd.h``; every function here has the
name of the C entry point it marshals arguments for.  All numerical work runs in the CUDA
library ``_build/librfdd.so`` (build it with ``paper_1711_09487_gb300.build.build()``).  There is
no CPU fallback: if the library is missing, loading fails with an error.

Dense arrays are numpy, row-major; complex data is numpy complex128 (interleaved re, im).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librfdd.so")

RFDD_OK = 0
RFDD_EINVAL = 1
RFDD_ENOTSYM = 2
RFDD_EPARTITION = 3
RFDD_ENOTSPD_M = 4
RFDD_ESINGULAR = 5
RFDD_ENOMEM = 6
RFDD_EADMIT = 7
RFDD_NOT_CONVERGED = 8
RFDD_ECUDA = 9
RFDD_ESTATE = 10
RFDD_FP64 = 0
RFDD_MIXED = 1
RFDD_MIDPOINT = 0
RFDD_GAUSS_LEGENDRE = 1

# Exported C symbols (kept in sync with include/rfdd.h; checked by tests/test_abi.py).
SYMBOLS = [
    "rfdd_default_options", "rfdd_last_error", "rfdd_status_string", "rfdd_quadrature", "rfdd_setup",
    "rfdd_layout", "rfdd_destroy", "rfdd_solve", "rfdd_result_get", "rfdd_result_info",
    "rfdd_result_pre_evals", "rfdd_result_free", "rfdd_factor", "rfdd_schur_copy", "rfdd_shifted_solve",
    "rfdd_filter_apply", "rfdd_lanczos", "rfdd_interior", "rfdd_rayleigh_ritz", "rfdd_solve_async",
    "rfdd_result_ready", "rfdd_memory_estimate", "rfdd_sym_eig", "rfdd_kernel_launches", "rfdd_profile",
    "rfdd_profile_get", "rfdd_profile_busy", "rfdd_cgemm", "rfdd_dgemm", "rfdd_cgemm_noalloc", "rfdd_inertia",
    "rfdd_polish", "rfdd_peak_probe", "rfdd_profile_bytes", "rfdd_release",
    "rfdd_server_default_options", "rfdd_server_create", "rfdd_server_add_pencil", "rfdd_server_submit",
    "rfdd_server_wait", "rfdd_server_submit_pencil", "rfdd_server_request_info", "rfdd_server_get_stats", "rfdd_server_remove_pencil",
    "rfdd_server_destroy", "rfdd_autotune", "rfdd_autotune_table",
    "rfdd_rfkrylov", "rfdd_set_interface_groups", "rfdd_interface_levels",
]


class RfddError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class rfdd_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("rowptr", C.POINTER(C.c_int64)), ("col", C.POINTER(C.c_int32)),
                ("val", C.POINTER(C.c_double)), ("location", C.c_int32)]


class rfdd_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("quad_rule", C.c_int), ("sigma", C.c_double), ("nev_b", C.c_int),
                ("psi", C.c_int), ("lanczos_tol", C.c_double), ("block", C.c_int), ("res_tol", C.c_double),
                ("max_passes", C.c_int), ("ir_max", C.c_int), ("seed", C.c_uint64), ("mem_budget", C.c_size_t),
                ("stream", C.c_void_p), ("guard_frac", C.c_double), ("min_guard", C.c_int),
                ("keep_schur", C.c_int), ("subspace_iters", C.c_int), ("m_align", C.c_int),
                ("pack_factors", C.c_int)]


class rfdd_info(C.Structure):
    _fields_ = [("nev", C.c_int64), ("mu", C.c_int64), ("k", C.c_int64), ("m", C.c_int64),
                ("passes", C.c_int32), ("ir_steps_max", C.c_int32), ("max_resid", C.c_double),
                ("pre_max_resid", C.c_double), ("pre_nev", C.c_int64), ("t_factor_ms", C.c_double),
                ("t_lanczos_ms", C.c_double), ("t_interior_ms", C.c_double), ("t_rr_ms", C.c_double),
                ("t_complete_ms", C.c_double), ("t_total_ms", C.c_double), ("status", C.c_int32),
                ("packed", C.c_int32), ("sigma", C.c_double), ("t_factor_enqueue_ms", C.c_double),
                ("factor_launches", C.c_int64), ("fp64_basis", C.c_int32), ("reserved0", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class rfdd_server_options(C.Structure):
    _fields_ = [("mem_budget", C.c_size_t), ("max_inflight", C.c_int32), ("max_bypass", C.c_int32),
                ("device", C.c_int32)]


class rfdd_request_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("pencil", C.c_int64), ("nev", C.c_int64), ("bytes", C.c_size_t),
                ("queue_ms", C.c_double), ("run_ms", C.c_double), ("latency_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class rfdd_server_stats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("failed", C.c_int64), ("waiting", C.c_int64),
                ("running", C.c_int32), ("peak_running", C.c_int32), ("in_use", C.c_size_t),
                ("peak_in_use", C.c_size_t), ("pencils", C.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing: run paper_1711_09487_gb300.build.build() first "
                           "(there is no CPU fallback)")
    lib = C.CDLL(p)
    vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double)
    lib.rfdd_last_error.restype = C.c_char_p
    lib.rfdd_status_string.restype = C.c_char_p
    lib.rfdd_status_string.argtypes = [C.c_int]
    lib.rfdd_default_options.argtypes = [C.POINTER(rfdd_options)]
    lib.rfdd_quadrature.argtypes = [C.c_double, C.c_double, i32, i32, dp, dp]
    lib.rfdd_setup.argtypes = [C.POINTER(rfdd_csr), C.POINTER(rfdd_csr), C.POINTER(C.c_int32), i32,
                               C.POINTER(rfdd_options), C.POINTER(vp)]
    lib.rfdd_layout.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32), C.POINTER(i64)]
    lib.rfdd_set_interface_groups.argtypes = [vp, i32, C.POINTER(i32)]
    lib.rfdd_interface_levels.argtypes = [vp, C.POINTER(i32), C.POINTER(i64)]
    lib.rfdd_destroy.argtypes = [vp]
    lib.rfdd_destroy.restype = None
    lib.rfdd_solve.argtypes = [vp, C.c_double, C.c_double, i32, C.POINTER(vp)]
    lib.rfdd_solve_async.argtypes = [vp, C.c_double, C.c_double, i32, vp, C.POINTER(vp)]
    lib.rfdd_rfkrylov.argtypes = [vp, C.c_double, C.c_double, i32, i64, C.POINTER(vp)]
    lib.rfdd_result_ready.argtypes = [vp]
    lib.rfdd_result_get.argtypes = [vp, C.POINTER(i64), C.POINTER(dp), C.POINTER(dp), C.POINTER(dp), i32]
    lib.rfdd_result_info.argtypes = [vp, C.POINTER(rfdd_info)]
    lib.rfdd_result_pre_evals.argtypes = [vp, C.POINTER(i64), dp]
    lib.rfdd_result_free.argtypes = [vp]
    lib.rfdd_result_free.restype = None
    lib.rfdd_factor.argtypes = [vp, i32, dp, dp]
    lib.rfdd_schur_copy.argtypes = [vp, i32, dp]
    lib.rfdd_shifted_solve.argtypes = [vp, i32, i32, i32, i64, dp, dp]
    lib.rfdd_filter_apply.argtypes = [vp, i64, dp, dp]
    lib.rfdd_lanczos.argtypes = [vp, i64, dp, C.POINTER(i64), dp, C.POINTER(i32)]
    lib.rfdd_interior.argtypes = [vp, C.c_double, i64, dp, C.POINTER(i64), C.POINTER(i64)]
    lib.rfdd_rayleigh_ritz.argtypes = [vp, i64, dp, C.POINTER(i64)]
    lib.rfdd_memory_estimate.argtypes = [vp, i32, i64, C.POINTER(C.c_size_t)]
    lib.rfdd_sym_eig.argtypes = [i64, dp, dp, dp]
    lib.rfdd_kernel_launches.restype = C.c_longlong
    fp = C.POINTER(C.c_float)
    lib.rfdd_cgemm.argtypes = [i64, i64, i64, fp, i64, fp, i64, fp, i64, C.c_double, C.c_double, i32]
    lib.rfdd_inertia.argtypes = [vp, C.c_double, C.POINTER(i64)]
    lib.rfdd_polish.argtypes = [vp, i64, dp, dp, dp]
    lib.rfdd_dgemm.argtypes = [i64, i64, i64, i32, dp, i64, i32, dp, i64, dp, i64, C.c_double, C.c_double, i32, i32]
    lib.rfdd_cgemm_noalloc.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, C.c_double, C.c_double, vp]
    lib.rfdd_profile.argtypes = [i32]
    lib.rfdd_profile_get.argtypes = [i32, C.POINTER(i64), dp, dp]
    lib.rfdd_profile_busy.argtypes = [i32, dp]
    lib.rfdd_peak_probe.argtypes = [i32, dp]
    lib.rfdd_profile_bytes.argtypes = [i32, dp]
    lib.rfdd_release.argtypes = [vp]
    lib.rfdd_autotune.argtypes = [i32]
    lib.rfdd_autotune_table.argtypes = [C.c_char_p, i64, C.POINTER(i64)]
    lib.rfdd_server_default_options.argtypes = [vp]
    lib.rfdd_server_default_options.restype = None
    lib.rfdd_server_create.argtypes = [vp, C.POINTER(vp)]
    lib.rfdd_server_add_pencil.argtypes = [vp, vp, vp, C.POINTER(i32), i32, vp, C.POINTER(i64)]
    lib.rfdd_server_submit.argtypes = [vp, i64, C.c_double, C.c_double, i32, i64, C.POINTER(i64)]
    lib.rfdd_server_wait.argtypes = [vp, i64, C.c_double, C.POINTER(i32), C.POINTER(vp)]
    lib.rfdd_server_submit_pencil.argtypes = [vp, vp, vp, C.POINTER(i32), i32, vp, C.c_double, C.c_double, i32,
                                              i64, C.POINTER(i64)]
    lib.rfdd_server_request_info.argtypes = [vp, i64, vp]
    lib.rfdd_server_get_stats.argtypes = [vp, vp]
    lib.rfdd_server_remove_pencil.argtypes = [vp, i64]
    lib.rfdd_server_destroy.argtypes = [vp]
    lib.rfdd_server_destroy.restype = None
    _lib = lib
    return lib


def _check(rc: int, ok=(RFDD_OK,)):
    if rc not in ok:
        lib = load()
        raise RfddError(rc, f"{lib.rfdd_status_string(rc).decode()}: {lib.rfdd_last_error().decode()}")
    return rc


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def rfdd_default_options(**overrides) -> rfdd_options:
    o = rfdd_options()
    load().rfdd_default_options(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def rfdd_status_string(code: int) -> str:
    return load().rfdd_status_string(code).decode()


def rfdd_quadrature(alpha: float, beta: float, n_nodes: int, rule: int = RFDD_MIDPOINT):
    z = np.zeros(2 * n_nodes)
    w = np.zeros(2 * n_nodes)
    _check(load().rfdd_quadrature(alpha, beta, n_nodes, rule, _dp(z), _dp(w)))
    return z.view(np.complex128), w.view(np.complex128)


class _Csr:
    """Keeps the arrays behind an rfdd_csr alive: numpy arrays (host), or CUDA torch tensors
    (int64 rowptr, int32 col, float64 val; the struct then says location = 1)."""

    def __init__(self, csr):
        if all(hasattr(getattr(csr, f), "data_ptr") and getattr(csr, f).is_cuda for f in ("rowptr", "col", "val")):
            import torch
            self.rowptr = csr.rowptr.contiguous().to(torch.int64)
            self.col = csr.col.contiguous().to(torch.int32)
            self.val = csr.val.contiguous().to(torch.float64)
            vp = lambda t, ty: C.cast(C.c_void_p(t.data_ptr()), C.POINTER(ty))
            self.s = rfdd_csr(int(self.rowptr.numel() - 1), vp(self.rowptr, C.c_int64), vp(self.col, C.c_int32),
                              vp(self.val, C.c_double), 1)
            return
        self.rowptr = np.ascontiguousarray(csr.rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(csr.col, dtype=np.int32)
        self.val = np.ascontiguousarray(csr.val, dtype=np.float64)
        self.s = rfdd_csr(int(len(self.rowptr) - 1), self.rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                          self.col.ctypes.data_as(C.POINTER(C.c_int32)), _dp(self.val), 0)


def _as_csr(x):
    if hasattr(x, "rowptr"):
        return x
    import scipy.sparse as sp
    a = sp.csr_matrix(x)
    a.sort_indices()

    class _T:
        pass
    t = _T()
    t.rowptr, t.col, t.val = a.indptr, a.indices, a.data
    return t


class Handle:
    """Owns an rfdd_handle* (destroyed with rfdd_destroy)."""

    def __init__(self, ptr, n, opts):
        self.ptr = C.c_void_p(ptr)
        self.n = n
        self.opts = opts

    def __del__(self):
        if getattr(self, "ptr", None) and self.ptr.value and _lib is not None:
            _lib.rfdd_destroy(self.ptr)
            self.ptr = C.c_void_p(None)

    close = __del__


def rfdd_setup(A, M, part, p: int, opts: rfdd_options | None = None) -> Handle:
    a, m = _Csr(_as_csr(A)), _Csr(_as_csr(M))
    pt = np.ascontiguousarray(part, dtype=np.int32)
    out = C.c_void_p()
    o = opts if opts is not None else rfdd_default_options()
    _check(load().rfdd_setup(C.byref(a.s), C.byref(m.s), pt.ctypes.data_as(C.POINTER(C.c_int32)), int(p),
                             C.byref(o), C.byref(out)))
    return Handle(out.value, a.s.n, o)


def rfdd_layout(h: Handle):
    lib = load()
    pp, ss = C.c_int32(), C.c_int64()
    _check(lib.rfdd_layout(h.ptr, None, None, C.byref(pp), C.byref(ss)))
    off = np.zeros(pp.value + 1, dtype=np.int64)
    perm = np.zeros(h.n, dtype=np.int64)
    _check(lib.rfdd_layout(h.ptr, off.ctypes.data_as(C.POINTER(C.c_int64)),
                           perm.ctypes.data_as(C.POINTER(C.c_int64)), None, None))
    return off, perm, int(ss.value)


def rfdd_set_interface_groups(h: Handle, group) -> None:
    """Two-level interface factorisation for these subdomain group labels (None: dense S)."""
    if group is None:
        _check(load().rfdd_set_interface_groups(h.ptr, 0, None))
        return
    g = np.ascontiguousarray(group, dtype=np.int32)
    ng = int(g.max()) + 1 if g.size else 0
    _check(load().rfdd_set_interface_groups(h.ptr, ng, g.ctypes.data_as(C.POINTER(C.c_int32))))


def rfdd_interface_levels(h: Handle):
    """(cls, s2): per interface unknown its level-1 group or -1, and the level-2 count."""
    lib = load()
    _, _, s = rfdd_layout(h)
    cls = np.zeros(s, dtype=np.int32)
    s2 = C.c_int64()
    _check(lib.rfdd_interface_levels(h.ptr, cls.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(s2)))
    return cls, int(s2.value)


class Result:
    def __init__(self, ptr, status, n):
        self.ptr = C.c_void_p(ptr)
        self.status = status
        self.n = n

    def __del__(self):
        if getattr(self, "ptr", None) and self.ptr.value and _lib is not None:
            _lib.rfdd_result_free(self.ptr)
            self.ptr = C.c_void_p(None)


def rfdd_solve(h: Handle, alpha: float, beta: float, n_nodes: int) -> Result:
    out = C.c_void_p()
    rc = load().rfdd_solve(h.ptr, alpha, beta, n_nodes, C.byref(out))
    _check(rc, ok=(RFDD_OK, RFDD_NOT_CONVERGED))
    return Result(out.value, rc, h.n)


def rfdd_rfkrylov(h: Handle, alpha: float, beta: float, n_nodes: int, max_dim: int = 0) -> Result:
    """RF-KRYLOV (Algorithm 1) on the handle's pencil, then the completion passes."""
    out = C.c_void_p()
    rc = load().rfdd_rfkrylov(h.ptr, alpha, beta, n_nodes, int(max_dim), C.byref(out))
    _check(rc, ok=(RFDD_OK, RFDD_NOT_CONVERGED))
    return Result(out.value, rc, h.n)


def rfdd_solve_async(h: Handle, alpha: float, beta: float, n_nodes: int, stream: int = 0) -> Result:
    out = C.c_void_p()
    _check(load().rfdd_solve_async(h.ptr, alpha, beta, n_nodes, C.c_void_p(stream or None), C.byref(out)))
    return Result(out.value, RFDD_OK, h.n)


def rfdd_result_ready(r: Result) -> int:
    return load().rfdd_result_ready(r.ptr)


def rfdd_result_get(r: Result, device: bool = False, vectors: bool = True):
    """Host copies (evals, evecs n x nev, resid); with device=True raw device pointers instead.
    vectors=False skips the eigenvector copy (evecs is then None)."""
    lib = load()
    nev = C.c_int64()
    ev, ex, rs = C.POINTER(C.c_double)(), C.POINTER(C.c_double)(), C.POINTER(C.c_double)()
    _check(lib.rfdd_result_get(r.ptr, C.byref(nev), C.byref(ev), C.byref(ex) if vectors else None, C.byref(rs),
                               1 if device else 0))
    k = nev.value
    if device:
        addr = lambda p: C.cast(p, C.c_void_p).value
        return k, addr(ev), addr(ex), addr(rs)
    evals = np.ctypeslib.as_array(ev, shape=(k,)).copy() if k else np.zeros(0)
    resid = np.ctypeslib.as_array(rs, shape=(k,)).copy() if k else np.zeros(0)
    if not vectors:
        return evals, None, resid
    evecs = (np.ctypeslib.as_array(ex, shape=(r.n * k,)).copy().reshape(r.n, k) if k
             else np.zeros((r.n, 0)))
    return evals, evecs, resid


def rfdd_result_info(r: Result) -> dict:
    inf = rfdd_info()
    _check(load().rfdd_result_info(r.ptr, C.byref(inf)))
    return inf.as_dict()


def rfdd_result_pre_evals(r: Result) -> np.ndarray:
    lib = load()
    cnt = C.c_int64()
    _check(lib.rfdd_result_pre_evals(r.ptr, C.byref(cnt), None))
    v = np.zeros(cnt.value)
    _check(lib.rfdd_result_pre_evals(r.ptr, C.byref(cnt), _dp(v)))
    return v


def rfdd_factor(h: Handle, z: np.ndarray, w: np.ndarray):
    z = np.ascontiguousarray(z, dtype=np.complex128)
    w = np.ascontiguousarray(w, dtype=np.complex128)
    _check(load().rfdd_factor(h.ptr, len(z), _dp(z.view(np.float64)), _dp(w.view(np.float64))))


def rfdd_schur_copy(h: Handle, node: int) -> np.ndarray:
    _, _, s = rfdd_layout(h)
    out = np.zeros((s, s), dtype=np.complex128)
    _check(load().rfdd_schur_copy(h.ptr, node, _dp(out.view(np.float64))))
    return out


def rfdd_shifted_solve(h: Handle, node: int, which: int, j: int, R: np.ndarray) -> np.ndarray:
    R = np.ascontiguousarray(R, dtype=np.complex128)
    if R.ndim == 1:
        R = R[:, None]
    X = np.zeros_like(R)
    _check(load().rfdd_shifted_solve(h.ptr, node, which, j, R.shape[1], _dp(R.view(np.float64)),
                                     _dp(X.view(np.float64))))
    return X


def rfdd_filter_apply(h: Handle, X: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    W = np.zeros_like(X)
    _check(load().rfdd_filter_apply(h.ptr, X.shape[1], _dp(X), _dp(W)))
    return W


def rfdd_lanczos(h: Handle, cap: int | None = None):
    lib = load()
    _, _, s = rfdd_layout(h)
    cap = cap or s
    Q = np.zeros((s, cap))
    tr = np.zeros(cap)
    mu, ns = C.c_int64(), C.c_int32()
    _check(lib.rfdd_lanczos(h.ptr, cap, _dp(Q), C.byref(mu), _dp(tr), C.byref(ns)))
    return Q[:, :mu.value].copy(), tr[:ns.value].copy()


def rfdd_interior(h: Handle, sigma: float = float("nan"), want_Z: bool = True):
    lib = load()
    k, kap = C.c_int64(), C.c_int64()
    _check(lib.rfdd_interior(h.ptr, sigma, 0, None, C.byref(k), C.byref(kap)))
    if not want_Z:
        return None, k.value, kap.value
    # the basis was built on the device by the call above; fetch it by a second call
    Z = np.zeros((h.n, k.value))
    _check(lib.rfdd_interior(h.ptr, sigma, k.value, _dp(Z), C.byref(k), C.byref(kap)))
    return Z, k.value, kap.value


def rfdd_rayleigh_ritz(h: Handle) -> np.ndarray:
    lib = load()
    k = C.c_int64()
    _check(lib.rfdd_rayleigh_ritz(h.ptr, 0, None, C.byref(k)))
    th = np.zeros(k.value)
    _check(lib.rfdd_rayleigh_ritz(h.ptr, k.value, _dp(th), C.byref(k)))
    return th


def rfdd_memory_estimate(h: Handle, n_nodes: int, nev_guess: int) -> int:
    b = C.c_size_t()
    _check(load().rfdd_memory_estimate(h.ptr, n_nodes, nev_guess, C.byref(b)))
    return int(b.value)


def rfdd_sym_eig(H: np.ndarray):
    """(evals ascending, evecs with eigenvector j in row j) of a dense symmetric FP64 matrix."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    n = H.shape[0]
    ev = np.zeros(n)
    V = np.zeros((n, n))
    _check(load().rfdd_sym_eig(n, _dp(H), _dp(ev), _dp(V)))
    return ev, V


def rfdd_cgemm(A: np.ndarray, B: np.ndarray, C: np.ndarray, alpha: float = 1.0, beta: float = 0.0,
               engine: int = 1) -> np.ndarray:
    """beta*C + alpha*A@B for complex64 row-major arrays on the GPU (engine 1: tensor cores)."""
    A = np.ascontiguousarray(A, dtype=np.complex64)
    B = np.ascontiguousarray(B, dtype=np.complex64)
    C = np.ascontiguousarray(C, dtype=np.complex64).copy()
    m, k = A.shape
    n = B.shape[1]
    fp = lambda x: x.view(np.float32).ctypes.data_as(C_float_p)
    _check(load().rfdd_cgemm(m, n, k, fp(A), k, fp(B), n, fp(C), n, alpha, beta, engine))
    return C


C_float_p = C.POINTER(C.c_float)
C_double_p = C.POINTER(C.c_double)


def rfdd_inertia(h: Handle, sigma: float) -> int:
    """Number of eigenvalues of (A, M) below sigma (Sylvester inertia through the DD blocks)."""
    c = C.c_int64()
    _check(load().rfdd_inertia(h.ptr, float(sigma), C.byref(c)))
    return int(c.value)


def rfdd_polish(h: Handle, lam, X):
    """Interior polish of approximate pairs: (lambda', X', resid) with X (n x nev, original
    ordering) keeping its interface rows and taking interior rows from the subdomain solves."""
    lam = np.ascontiguousarray(lam, dtype=np.float64).copy()
    X = np.ascontiguousarray(X, dtype=np.float64).copy()
    if X.ndim != 2 or X.shape[0] != h.n or X.shape[1] != lam.shape[0]:
        raise ValueError("rfdd_polish: X must be n x nev with nev = len(lam)")
    nev = lam.shape[0]
    res = np.zeros(nev)
    fp = lambda a: a.ctypes.data_as(C_double_p)
    _check(load().rfdd_polish(h.ptr, nev, fp(lam), fp(X), fp(res)))
    return lam, X, res


def rfdd_dgemm(A: np.ndarray, B: np.ndarray, C: np.ndarray, alpha: float = 1.0, beta: float = 0.0,
               ta: bool = False, tb: bool = False, engine: int = 1, sym: bool = False) -> np.ndarray:
    """beta*C + alpha*op(A)@op(B) for float64 row-major arrays on the GPU (engine 1: double-FP32)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    C = np.array(C, dtype=np.float64, order="C", copy=True)
    m, n = C.shape
    k = A.shape[0] if ta else A.shape[1]
    lda, ldb = A.shape[1], B.shape[1]
    dptr = lambda X: X.ctypes.data_as(C_double_p)
    _check(load().rfdd_dgemm(m, n, k, int(ta), dptr(A), lda, int(tb), dptr(B), ldb, dptr(C), n, alpha, beta,
                             engine, int(sym)))
    return C


def rfdd_cgemm_noalloc(m: int, n: int, k: int, A_ptr: int, lda: int, B_ptr: int, ldb: int, C_ptr: int, ldc: int,
                       alpha: float = 1.0, beta: float = 0.0, stream: int = 0):
    """Allocation-free tensor-core GEMM on device pointers (complex64, row-major); see rfdd.h."""
    _check(load().rfdd_cgemm_noalloc(m, n, k, C.c_void_p(A_ptr), lda, C.c_void_p(B_ptr), ldb, C.c_void_p(C_ptr), ldc,
                                     alpha, beta, C.c_void_p(stream or None)))


def rfdd_peak_probe(which: int) -> float:
    """TFLOP/s of one arithmetic unit on the current device: 0 the tensor pipe's TF32 MMA rate,
    1 FP64 FMA, 2 FP32 FMA (CUDA cores), 3 a plain TF32 8192^3 GEMM through the tensor-core kernel."""
    t = C.c_double()
    _check(load().rfdd_peak_probe(int(which), C.byref(t)))
    return float(t.value)


def rfdd_autotune(mode: int) -> int:
    """Tile-shape autotuner: 0 off (fixed rule), 1 on, 2 forget every class.  Returns whether it
    was on."""
    r = load().rfdd_autotune(int(mode))
    if r < 0:
        _check(-r)
    return r


def rfdd_autotune_table() -> list[dict]:
    """The autotuner's classes: key, winner (-1 undecided; 0 one-CTA, 1 two-CTA) and the mean
    milliseconds per GFLOP each candidate measured."""
    lib = load()
    n = C.c_int64()
    _check(lib.rfdd_autotune_table(None, 0, C.byref(n)))
    buf = C.create_string_buffer(n.value + 1)
    _check(lib.rfdd_autotune_table(buf, n.value + 1, C.byref(n)))
    out = []
    for line in buf.value.decode().splitlines():
        f = line.split()
        out.append({"device": int(f[0]), "complex": int(f[1]), "splits": int(f[2]), "kbucket": int(f[3]),
                    "tbucket": int(f[4]), "winner": int(f[5]), "n": [int(f[6]), int(f[8])],
                    "ms_per_gflop": [float(f[7]), float(f[9])]})
    return out


def rfdd_profile_bytes(kind: int) -> float:
    """Model (compulsory) DRAM bytes of the recorded launches of one kind."""
    b = C.c_double()
    _check(load().rfdd_profile_bytes(int(kind), C.byref(b)))
    return float(b.value)


def rfdd_release(h: Handle):
    """Free the factors and solve buffers of the handle's last solve (its set-up stays)."""
    _check(load().rfdd_release(h.ptr))


def rfdd_server_default_options(**overrides) -> rfdd_server_options:
    o = rfdd_server_options()
    load().rfdd_server_default_options(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


class Server:
    """Owns an rfdd_server* (continuous batching of interval requests on one GPU)."""

    def __init__(self, **opts):
        lib = load()
        self.opts = rfdd_server_default_options(**opts)
        out = C.c_void_p()
        _check(lib.rfdd_server_create(C.byref(self.opts), C.byref(out)))
        self.ptr = out
        self.n_of = {}    # pencil id -> n
        self.n_req = {}   # request id -> n, for requests that brought their own pencil

    def add_pencil(self, A, M, part, p: int, opts: rfdd_options | None = None) -> int:
        a, m = _Csr(_as_csr(A)), _Csr(_as_csr(M))
        pt = np.ascontiguousarray(part, dtype=np.int32)
        o = opts if opts is not None else rfdd_default_options()
        pid = C.c_int64()
        _check(load().rfdd_server_add_pencil(self.ptr, C.byref(a.s), C.byref(m.s),
                                             pt.ctypes.data_as(C.POINTER(C.c_int32)), int(p), C.byref(o),
                                             C.byref(pid)))
        self.n_of[pid.value] = a.s.n
        return pid.value

    def submit(self, pencil: int, alpha: float, beta: float, n_nodes: int, nev_hint: int = 0) -> int:
        rid = C.c_int64()
        _check(load().rfdd_server_submit(self.ptr, int(pencil), float(alpha), float(beta), int(n_nodes),
                                         int(nev_hint), C.byref(rid)))
        return rid.value

    def submit_pencil(self, A, M, part, p: int, alpha: float, beta: float, n_nodes: int, nev_hint: int = 0,
                      opts: rfdd_options | None = None) -> int:
        """Queue a request that brings its own pencil (set up, solved and freed by the server)."""
        a, m = _Csr(_as_csr(A)), _Csr(_as_csr(M))
        pt = np.ascontiguousarray(part, dtype=np.int32)
        o = opts if opts is not None else rfdd_default_options()
        rid = C.c_int64()
        _check(load().rfdd_server_submit_pencil(self.ptr, C.byref(a.s), C.byref(m.s),
                                                pt.ctypes.data_as(C.POINTER(C.c_int32)), int(p), C.byref(o),
                                                float(alpha), float(beta), int(n_nodes), int(nev_hint),
                                                C.byref(rid)))
        self.n_req[rid.value] = a.s.n
        return rid.value

    def wait(self, request: int, timeout_ms: float = -1.0):
        """Result of a finished request (None while it runs); raises if its solve failed."""
        done, out = C.c_int32(), C.c_void_p()
        _check(load().rfdd_server_wait(self.ptr, int(request), float(timeout_ms), C.byref(done), C.byref(out)))
        if not done.value:
            return None
        info = self.request_info(request)
        if out.value is None:
            raise RfddError(info["status"], f"request {request} failed: {rfdd_status_string(info['status'])}")
        n = self.n_req.pop(request, None) or self.n_of[info["pencil"]]
        return Result(out.value, info["status"], n)

    def request_info(self, request: int) -> dict:
        inf = rfdd_request_info()
        _check(load().rfdd_server_request_info(self.ptr, int(request), C.byref(inf)))
        return inf.as_dict()

    def stats(self) -> dict:
        st = rfdd_server_stats()
        _check(load().rfdd_server_get_stats(self.ptr, C.byref(st)))
        return st.as_dict()

    def remove_pencil(self, pencil: int):
        _check(load().rfdd_server_remove_pencil(self.ptr, int(pencil)))

    def close(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value and _lib is not None:
            _lib.rfdd_server_destroy(self.ptr)
            self.ptr = C.c_void_p(None)

    __del__ = close


def rfdd_kernel_launches() -> int:
    return int(load().rfdd_kernel_launches())


def rfdd_profile(enable: bool):
    _check(load().rfdd_profile(1 if enable else 0))


def rfdd_profile_get(kind: int):
    """(launches, milliseconds, algorithmic flops) recorded for one kernel kind."""
    n, ms, fl = C.c_int64(), C.c_double(), C.c_double()
    _check(load().rfdd_profile_get(kind, C.byref(n), C.byref(ms), C.byref(fl)))
    return n.value, ms.value, fl.value


def rfdd_profile_busy(kind: int) -> float:
    """Milliseconds during which at least one recorded launch of this kind was running."""
    ms = C.c_double()
    _check(load().rfdd_profile_busy(kind, C.byref(ms)))
    return ms.value


def solve(A, M, part, p, alpha, beta, n_nodes, groups=None, **opts):
    """Convenience: setup + solve + host results (evals, evecs in original order, resid, info).
    ``groups``: subdomain group labels for the two-level interface factorisation."""
    h = rfdd_setup(A, M, part, p, rfdd_default_options(**opts))
    if groups is not None:
        rfdd_set_interface_groups(h, groups)
    r = rfdd_solve(h, alpha, beta, n_nodes)
    ev, X, rs = rfdd_result_get(r)
    return ev, X, rs, rfdd_result_info(r)
