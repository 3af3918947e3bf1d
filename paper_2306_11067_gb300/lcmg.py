"""ctypes binding of liblcmg.so (declared in include/lcmg.h).

Argument marshalling only: every function calls the C entry point of the
same name; all arithmetic runs in the library's CUDA kernels.  Host arrays
are numpy arrays; device buffers are torch CUDA tensors (passed by their
data pointers).  A missing library raises at import of this module's
``lib()``; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblcmg.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lcmg.h")

LCMG_OK, LCMG_ERR_INVALID_ARG, LCMG_ERR_NOMEM, LCMG_ERR_CUDA = 0, 1, 2, 3
LCMG_ERR_NOT_READY, LCMG_ERR_CANCELLED, LCMG_ERR_STATE = 4, 5, 6
CONVERGED, MAXIT, BREAKDOWN, NONFINITE = 0, 1, 2, 3
SMOOTH_L1_JACOBI, SMOOTH_JACOBI = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
MODE_BATCHED, MODE_SEQUENTIAL = 0, 1


class LcmgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lcmg status {status}: {msg}")
        self.status = status


class lcmg_params(C.Structure):
    _fields_ = [("levels", C.c_int32), ("coarse_max", C.c_int32), ("nu", C.c_int32),
                ("smoother", C.c_int32), ("omega", C.c_double), ("q", C.c_double),
                ("d_min", C.c_double), ("tol", C.c_double), ("maxit", C.c_int32),
                ("precision", C.c_int32), ("mode", C.c_int32), ("check_every", C.c_int32),
                ("graphs", C.c_int32), ("timing", C.c_int32),
                ("vfuse", C.c_int32),
                ("keep_direction", C.c_int32),
                ("autotune", C.c_int32),
                ("spmv_variant", C.c_int32),
                ("stop_rule", C.c_int32),
                ("precond", C.c_int32), ("gmres_restart", C.c_int32),
                ("coarsening", C.c_int32), ("amg_coarse_max", C.c_int32), ("compact_cols", C.c_int32),
                ("alpha_fuse", C.c_int32), ("beta_fuse", C.c_int32),
                ("spmv_variant_at", C.c_int32), ("max_blocks", C.c_int32),
                ("smoother_fp16", C.c_int32)]


class lcmg_stats(C.Structure):
    _fields_ = [("column_iterations", C.c_int64), ("batch_iterations", C.c_int64),
                ("kernel_launches", C.c_int64), ("iterate_ms", C.c_double),
                ("op_ms_a", C.c_double), ("op_ms_at", C.c_double),
                ("op_launches", C.c_int64), ("op_bytes", C.c_int64),
                ("tuned_spmv_a", C.c_int32), ("tuned_spmv_at", C.c_int32), ("tuned_vfuse", C.c_int32),
                ("vcycle_ms", C.c_double), ("vcycle_count", C.c_int64), ("vcycle_bytes", C.c_int64)]


class lcmg_problem(C.Structure):
    _fields_ = [("n_v", C.c_int32), ("n_h", C.c_int32), ("kind", C.c_int32), ("m", C.c_int64),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p), ("val_dtype", C.c_int32),
                ("kh", C.c_int32), ("kw", C.c_int32), ("psf", C.c_void_p)]


class lcmg_request(C.Structure):
    _fields_ = [("problem", C.c_int32), ("n_lambda", C.c_int32), ("lambda_", C.c_void_p), ("b", C.c_void_p),
                ("tol", C.c_double), ("max_outer", C.c_int32), ("warm", C.c_int32)]


class lcmg_result(C.Structure):
    _fields_ = [("state", C.c_int32), ("n_lambda", C.c_int32), ("n_outer", C.c_int32),
                ("n_solves", C.c_int64), ("n_converged", C.c_int64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("x", C.c_void_p), ("rho", C.c_void_p), ("eta", C.c_void_p), ("iters", C.c_void_p),
                ("status", C.c_void_p), ("history", C.c_void_p)]


class lcmg_server_stats(C.Structure):
    _fields_ = [("resident_bytes", C.c_size_t), ("contexts", C.c_int32), ("pending", C.c_int32),
                ("running", C.c_int32), ("peak_running", C.c_int32), ("admitted", C.c_int64),
                ("completed", C.c_int64), ("evictions", C.c_int64), ("reuses", C.c_int64)]


_lib = None
_P = C.c_void_p
_I32 = C.c_int32
_I64 = C.c_int64
_D = C.c_double
_PD = C.POINTER(C.c_double)
_PI32 = C.POINTER(C.c_int32)
_PI64 = C.POINTER(C.c_int64)

_SIGS = {
    "lcmg_default_params": (None, [C.POINTER(lcmg_params)]),
    "lcmg_last_error": (C.c_char_p, []),
    "lcmg_version": (C.c_char_p, []),
    "lcmg_create": (C.c_int, [C.POINTER(_P), C.c_int, _P, C.POINTER(lcmg_params)]),
    "lcmg_destroy": (C.c_int, [_P]),
    "lcmg_set_params": (C.c_int, [_P, C.POINTER(lcmg_params)]),
    "lcmg_set_grid": (C.c_int, [_P, _I32, _I32]),
    "lcmg_set_forward_csr": (C.c_int, [_P, _I64, _I64, _P, _P, _P, _I32]),
    "lcmg_set_forward_stencil": (C.c_int, [_P, _I32, _I32, _P]),
    "lcmg_set_forward_separable": (C.c_int, [_P, _I32, _P, _I32, _P]),
    "lcmg_forward_form": (C.c_int, [_P, _PI32]),
    "lcmg_set_weights": (C.c_int, [_P, _P, _I64]),
    "lcmg_set_weights_dev": (C.c_int, [_P, _P, _I64]),
    "lcmg_get_weights": (C.c_int, [_P, _P, _I64]),
    "lcmg_solve": (C.c_int, [_P, _I32, _P, _I32, _P, _P, _P, _P, _P, _P, _P]),
    "lcmg_solve_dev": (C.c_int, [_P, _I32, _P, _I32, _P, _P, _P, _P, _P, _P, _P]),
    "lcmg_lcurve_corner": (C.c_int, [_I32, _P, _P, _PI32]),
    "lcmg_update_weights": (C.c_int, [_P, _P, _D, _D, _P]),
    "lcmg_update_weights_dev": (C.c_int, [_P, _P, _D, _D]),
    "lcmg_cull_lambdas": (C.c_int, [_I32, _I32, _PI32, _PI32]),
    "lcmg_rs_split": (C.c_int, [_I64, _P, _P, _P, _D, _P]),
    "lcmg_rs_interp": (C.c_int, [_I64, _P, _P, _P, _D, _P, _I64, _P, _P, _P, _PI64]),
    "lcmg_amg_levels": (C.c_int, [_P, _I32, _P, _PI32]),
    "lcmg_pmis_split": (C.c_int, [_I64, _P, _P, _P, _D, C.c_uint64, _P]),
    "lcmg_lcurve_run": (C.c_int, [_P, _I32, _P, _P, _I32, _P, _P, _PI32, _PI64, _PI64]),
    "lcmg_lcurve_run_dev": (C.c_int, [_P, _I32, _P, _P, _I32, _P, _P, _PI32, _PI64, _PI64]),
    "lcmg_get_stats": (C.c_int, [_P, C.POINTER(lcmg_stats)]),
    "lcmg_apply_normal_dev": (C.c_int, [_P, _I32, _P, _P, _P]),
    "lcmg_apply_vcycle_dev": (C.c_int, [_P, _I32, _P, _P, _P]),
    "lcmg_get_level": (C.c_int, [_P, _I32, _PI32, _PI32, _P, _P]),
    "lcmg_num_levels": (C.c_int, [_P, _PI32]),
    "lcmg_get_diag": (C.c_int, [_P, _P]),
    "lcmg_fma_peak": (C.c_int, [C.c_int, _I32, _PD]),
    "lcmg_apply_normal_noalloc": (C.c_int, [C.c_int, _P, _I32, _I32, _I64, _P, _P, _P, _P, _P, _P, _I32, _P,
                                            _I32, _P, _P, _P]),
    "lcmg_server_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_size_t, _I32, C.POINTER(lcmg_params)]),
    "lcmg_server_add_problem": (C.c_int, [_P, C.POINTER(lcmg_problem), _PI32]),
    "lcmg_server_submit": (C.c_int, [_P, C.POINTER(lcmg_request), C.POINTER(C.c_uint64)]),
    "lcmg_server_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(lcmg_result)]),
    "lcmg_server_wait": (C.c_int, [_P, C.c_uint64, _D, C.POINTER(lcmg_result)]),
    "lcmg_server_cancel": (C.c_int, [_P, C.c_uint64]),
    "lcmg_server_get_stats": (C.c_int, [_P, C.POINTER(lcmg_server_stats)]),
    "lcmg_server_footprint": (C.c_int, [_P, _I32, _I32, C.POINTER(C.c_size_t)]),
    "lcmg_server_last_error": (C.c_char_p, []),
    "lcmg_server_destroy": (C.c_int, [_P]),
}


def lib() -> C.CDLL:
    """Load liblcmg.so (fails loudly if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2306_11067_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/lcmg.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lcmg_\w+)\s*\(", txt, re.M)))


def _check(st: int):
    if st != LCMG_OK:
        raise LcmgError(st, lib().lcmg_last_error().decode())


def _ptr(a) -> int | None:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
def lcmg_default_params() -> lcmg_params:
    p = lcmg_params()
    lib().lcmg_default_params(C.byref(p))
    return p


def lcmg_version() -> str:
    return lib().lcmg_version().decode()


def lcmg_last_error() -> str:
    return lib().lcmg_last_error().decode()


def lcmg_create(device: int = 0, stream=None, params: lcmg_params | None = None):
    h = _P()
    s = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().lcmg_create(C.byref(h), device, s, C.byref(params) if params is not None else None))
    return h


def lcmg_destroy(ctx):
    _check(lib().lcmg_destroy(ctx))


def lcmg_set_params(ctx, params: lcmg_params):
    _check(lib().lcmg_set_params(ctx, C.byref(params)))


def lcmg_set_grid(ctx, n_v: int, n_h: int):
    _check(lib().lcmg_set_grid(ctx, n_v, n_h))


def lcmg_set_forward_csr(ctx, m, n, row_ptr, col, val):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    if val.dtype == np.float32:
        va, dt = np.ascontiguousarray(val), 0
    else:
        va, dt = _f64(val), 1
    _check(lib().lcmg_set_forward_csr(ctx, m, n, _ptr(rp), _ptr(ci), _ptr(va), dt))


def lcmg_set_forward_stencil(ctx, psf):
    p = _f64(psf)
    _check(lib().lcmg_set_forward_stencil(ctx, p.shape[0], p.shape[1], _ptr(p)))


def lcmg_set_forward_separable(ctx, fv, fh):
    a, b = _f64(fv), _f64(fh)
    _check(lib().lcmg_set_forward_separable(ctx, a.size, _ptr(a), b.size, _ptr(b)))


FORM_NONE, FORM_CSR, FORM_PSF2D, FORM_SEPARABLE = 0, 1, 2, 3


def lcmg_forward_form(ctx) -> int:
    f = C.c_int32(0)
    _check(lib().lcmg_forward_form(ctx, C.byref(f)))
    return int(f.value)


def lcmg_set_weights(ctx, d):
    d = _f64(d)
    _check(lib().lcmg_set_weights(ctx, _ptr(d), d.size))


def lcmg_set_weights_dev(ctx, d_dev, n_edges: int):
    _check(lib().lcmg_set_weights_dev(ctx, _ptr(d_dev), n_edges))


def lcmg_get_weights(ctx, n_edges: int):
    out = np.empty(n_edges)
    _check(lib().lcmg_get_weights(ctx, _ptr(out), n_edges))
    return out


def lcmg_solve(ctx, lambdas, b, x0=None):
    """b: (n_rhs, m) or (m,); returns x (n_rhs, n_lambda, n), rho, eta, iters, status."""
    lam = _f64(lambdas)
    b2 = _f64(np.atleast_2d(b))
    nr, nl = b2.shape[0], lam.size
    n = _solve_n(ctx, x0, b2)
    x = np.empty((nr, nl, n))
    rho, eta = np.empty((nr, nl)), np.empty((nr, nl))
    its, st = np.empty((nr, nl), np.int32), np.empty((nr, nl), np.int32)
    x0a = None if x0 is None else _f64(x0)
    _check(lib().lcmg_solve(ctx, nl, _ptr(lam), nr, _ptr(b2), _ptr(x0a), _ptr(x), _ptr(rho),
                            _ptr(eta), _ptr(its), _ptr(st)))
    return dict(x=x, rho=rho, eta=eta, iters=its, status=st)


_N_CACHE: dict = {}


def _solve_n(ctx, x0, b2):
    key = ctx.value
    if key in _N_CACHE:
        return _N_CACHE[key]
    raise LcmgError(LCMG_ERR_STATE, "grid size unknown to the binding: call lcmg_set_grid through it")


def lcmg_solve_dev(ctx, lambdas, b_dev, x_dev, x0_dev=None, rho_dev=None, eta_dev=None,
                   iters_dev=None, status_dev=None):
    lam = _f64(lambdas)
    nr = b_dev.shape[0] if b_dev.dim() == 2 else 1
    _check(lib().lcmg_solve_dev(ctx, lam.size, _ptr(lam), nr, _ptr(b_dev), _ptr(x0_dev), _ptr(x_dev),
                                _ptr(rho_dev), _ptr(eta_dev), _ptr(iters_dev), _ptr(status_dev)))


def lcmg_lcurve_corner(rho, eta) -> int:
    r, e = _f64(rho), _f64(eta)
    idx = C.c_int32()
    _check(lib().lcmg_lcurve_corner(r.size, _ptr(r), _ptr(e), C.byref(idx)))
    return idx.value


def lcmg_update_weights(ctx, x_star, q, d_min, n_edges: int):
    xs = _f64(x_star)
    d = np.empty(n_edges)
    _check(lib().lcmg_update_weights(ctx, _ptr(xs), q, d_min, _ptr(d)))
    return d


def lcmg_update_weights_dev(ctx, x_star_dev, q, d_min):
    _check(lib().lcmg_update_weights_dev(ctx, _ptr(x_star_dev), q, d_min))


def lcmg_cull_lambdas(m: int, i_prev: int):
    lo, hi = C.c_int32(), C.c_int32()
    _check(lib().lcmg_cull_lambdas(m, i_prev, C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def _csr_in(K):
    """(n, row_ptr int64, col int32 sorted per row, val f64) of a square
    scipy-like CSR matrix."""
    n = K.shape[0]
    K = K.tocsr()
    K.sort_indices()
    return (n, np.ascontiguousarray(K.indptr, dtype=np.int64), np.ascontiguousarray(K.indices, dtype=np.int32),
            np.ascontiguousarray(K.data, dtype=np.float64))


def lcmg_rs_split(K, theta=0.25):
    """C/F split of classical AMG (host): int8 array, 1 = C, 0 = F."""
    n, rp, ci, v = _csr_in(K)
    cf = np.empty(n, np.int8)
    _check(lib().lcmg_rs_split(n, _ptr(rp), _ptr(ci), _ptr(v), theta, _ptr(cf)))
    return cf


def lcmg_rs_interp(K, cf, theta=0.25):
    """Interpolation of the split cf (host): (row_ptr, col, val, n_coarse)."""
    n, rp, ci, v = _csr_in(K)
    cf = np.ascontiguousarray(cf, dtype=np.int8)
    nnz = C.c_int64()
    prp = np.empty(n + 1, np.int64)
    cap = int(v.size) + n
    pci = np.empty(cap, np.int32)
    pv = np.empty(cap)
    _check(lib().lcmg_rs_interp(n, _ptr(rp), _ptr(ci), _ptr(v), theta, _ptr(cf), cap, _ptr(prp), _ptr(pci),
                                _ptr(pv), C.byref(nnz)))
    return prp, pci[:nnz.value].copy(), pv[:nnz.value].copy(), int(cf.sum())


def lcmg_pmis_split(K, seed, theta=0.25):
    """PMIS C/F split on the current device: int8 array, 1 = C, 0 = F."""
    n, rp, ci, v = _csr_in(K)
    cf = np.empty(n, np.int8)
    _check(lib().lcmg_pmis_split(n, _ptr(rp), _ptr(ci), _ptr(v), theta, seed, _ptr(cf)))
    return cf


def lcmg_amg_levels(ctx):
    sizes = np.zeros(64, np.int64)
    nl = C.c_int32()
    _check(lib().lcmg_amg_levels(ctx, 64, _ptr(sizes), C.byref(nl)))
    return sizes[:nl.value].copy()


def lcmg_lcurve_run(ctx, lambdas, b, max_outer: int, n: int):
    lam = _f64(lambdas)
    bb = _f64(b)
    x = np.empty(n)
    hist = np.zeros(max_outer, np.int32)
    no, ns, nc = C.c_int32(), C.c_int64(), C.c_int64()
    _check(lib().lcmg_lcurve_run(ctx, lam.size, _ptr(lam), _ptr(bb), max_outer, _ptr(x), _ptr(hist),
                                 C.byref(no), C.byref(ns), C.byref(nc)))
    return dict(x=x, history=list(hist[:no.value]), n_solves=ns.value, n_converged=nc.value)


def lcmg_lcurve_run_dev(ctx, lambdas, b_dev, max_outer: int, x_out_dev):
    lam = _f64(lambdas)
    hist = np.zeros(max_outer, np.int32)
    no, ns, nc = C.c_int32(), C.c_int64(), C.c_int64()
    _check(lib().lcmg_lcurve_run_dev(ctx, lam.size, _ptr(lam), _ptr(b_dev), max_outer, _ptr(x_out_dev),
                                     _ptr(hist), C.byref(no), C.byref(ns), C.byref(nc)))
    return dict(history=list(hist[:no.value]), n_solves=ns.value, n_converged=nc.value)


def lcmg_get_stats(ctx) -> dict:
    s = lcmg_stats()
    _check(lib().lcmg_get_stats(ctx, C.byref(s)))
    return {k: getattr(s, k) for k, _ in s._fields_}


def lcmg_apply_normal_dev(ctx, lambdas, x_dev, y_dev):
    lam = _f64(lambdas)
    _check(lib().lcmg_apply_normal_dev(ctx, lam.size, _ptr(lam), _ptr(x_dev), _ptr(y_dev)))


def lcmg_apply_vcycle_dev(ctx, lambdas, r_dev, z_dev):
    lam = _f64(lambdas)
    _check(lib().lcmg_apply_vcycle_dev(ctx, lam.size, _ptr(lam), _ptr(r_dev), _ptr(z_dev)))


def lcmg_num_levels(ctx) -> int:
    v = C.c_int32()
    _check(lib().lcmg_num_levels(ctx, C.byref(v)))
    return v.value


def lcmg_get_level(ctx, k: int):
    nv, nh = C.c_int32(), C.c_int32()
    _check(lib().lcmg_get_level(ctx, k, C.byref(nv), C.byref(nh), None, None))
    n = nv.value * nh.value
    gl, ga = np.empty((25, n)), np.empty((25, n))
    if k > 0:
        _check(lib().lcmg_get_level(ctx, k, None, None, _ptr(gl), _ptr(ga)))
    return nv.value, nh.value, gl, ga


def lcmg_apply_normal_noalloc(device, stream, n_v, n_h, m, row_ptr, col, val, row_ptr_t, col_t, val_t,
                              d, lambdas, p, q):
    """Allocation-free q = (A^T A + lambda^2 L^T D^2 L) p; every array is a
    torch CUDA tensor on `device` except ``lambdas`` (host).  For callers
    that cannot allocate device memory at the point of use."""
    lam = _f64(lambdas)
    dt = 0 if str(val.dtype).endswith("float32") else 1
    s = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().lcmg_apply_normal_noalloc(device, s, n_v, n_h, m, _ptr(row_ptr), _ptr(col), _ptr(val),
                                           _ptr(row_ptr_t), _ptr(col_t), _ptr(val_t), dt, _ptr(d), lam.size,
                                           _ptr(lam), _ptr(p), _ptr(q)))


def lcmg_fma_peak(device: int, precision: int) -> float:
    """Measured FP64 (PREC_FP64) or FP32 (PREC_MIXED) multiply-add peak, TFLOP/s."""
    v = C.c_double(0.0)
    _check(lib().lcmg_fma_peak(device, precision, C.byref(v)))
    return float(v.value)


def lcmg_get_diag(ctx, n: int):
    out = np.empty(n)
    _check(lib().lcmg_get_diag(ctx, _ptr(out)))
    return out


# ---------------------------------------------------------------------------
class Solver:
    """Convenience owner of one context (same calls, bound to it)."""

    def __init__(self, n_v, n_h, device=0, stream=None, **params):
        p = lcmg_default_params()
        for k, v in params.items():
            setattr(p, k, v)
        self.params = p
        self.ctx = lcmg_create(device, stream, p)
        self.n_v, self.n_h = n_v, n_h
        self.n = n_v * n_h
        self.n_edges = n_h * (n_v - 1) + (n_h - 1) * n_v
        lcmg_set_grid(self.ctx, n_v, n_h)
        _N_CACHE[self.ctx.value] = self.n

    def set_params(self, **params):
        for k, v in params.items():
            setattr(self.params, k, v)
        lcmg_set_params(self.ctx, self.params)

    def set_forward_csr(self, A):
        lcmg_set_forward_csr(self.ctx, A.m, A.n, A.row_ptr, A.col, A.val)

    def set_forward_stencil(self, psf):
        lcmg_set_forward_stencil(self.ctx, psf)

    def set_forward_separable(self, fv, fh):
        lcmg_set_forward_separable(self.ctx, fv, fh)

    def forward_form(self):
        return lcmg_forward_form(self.ctx)

    def set_weights(self, d):
        lcmg_set_weights(self.ctx, d)

    def solve(self, lambdas, b, x0=None):
        return lcmg_solve(self.ctx, lambdas, b, x0)

    def update_weights(self, x_star, q=2.0, d_min=1e-3):
        return lcmg_update_weights(self.ctx, x_star, q, d_min, self.n_edges)

    def lcurve_run(self, lambdas, b, max_outer=15):
        return lcmg_lcurve_run(self.ctx, lambdas, b, max_outer, self.n)

    def stats(self):
        return lcmg_get_stats(self.ctx)

    def close(self):
        if self.ctx:
            _N_CACHE.pop(self.ctx.value, None)
            lcmg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
def _scheck(st: int):
    if st != LCMG_OK:
        raise LcmgError(st, lib().lcmg_server_last_error().decode())


class Server:
    """Serving front end: lcmg_server_* (admission by HBM footprint, slot
    threads with their own contexts and streams, resident operators)."""

    def __init__(self, device=0, hbm_budget=8 << 30, slots=4, **params):
        p = lcmg_default_params()
        for k, v in params.items():
            setattr(p, k, v)
        self.params = p
        h = _P()
        _scheck(lib().lcmg_server_create(C.byref(h), device, int(hbm_budget), slots, C.byref(p)))
        self.h = h
        self._probs = {}
        self._reqs = {}

    def add_csr(self, n_v, n_h, A):
        rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(A.col, dtype=np.int32)
        if A.val.dtype == np.float32:
            va, dt = np.ascontiguousarray(A.val), 0
        else:
            va, dt = _f64(A.val), 1
        pr = lcmg_problem(n_v=n_v, n_h=n_h, kind=0, m=A.m, row_ptr=_ptr(rp), col=_ptr(ci), val=_ptr(va),
                          val_dtype=dt)
        i = C.c_int32()
        _scheck(lib().lcmg_server_add_problem(self.h, C.byref(pr), C.byref(i)))
        self._probs[i.value] = (n_v * n_h, A.m)
        return i.value

    def add_psf(self, n_v, n_h, psf):
        p = _f64(psf)
        pr = lcmg_problem(n_v=n_v, n_h=n_h, kind=1, m=n_v * n_h, kh=p.shape[0], kw=p.shape[1], psf=_ptr(p))
        i = C.c_int32()
        _scheck(lib().lcmg_server_add_problem(self.h, C.byref(pr), C.byref(i)))
        self._probs[i.value] = (n_v * n_h, n_v * n_h)
        return i.value

    def submit(self, problem, lambdas, b, tol=0.0, max_outer=0, warm=0):
        lam = _f64(lambdas)
        bb = _f64(b)
        rq = lcmg_request(problem=problem, n_lambda=lam.size, lambda_=_ptr(lam), b=_ptr(bb), tol=tol,
                          max_outer=max_outer, warm=warm)
        t = C.c_uint64()
        _scheck(lib().lcmg_server_submit(self.h, C.byref(rq), C.byref(t)))
        self._reqs[t.value] = (problem, lam.size, max_outer)
        return t.value

    def _result(self, ticket, fn):
        problem, nl, mo = self._reqs[ticket]
        n, _ = self._probs[problem]
        x = np.empty((nl, n) if mo == 0 else n)
        rho, eta = np.empty(nl), np.empty(nl)
        its, st = np.empty(nl, np.int32), np.empty(nl, np.int32)
        hist = np.zeros(max(mo, 1), np.int32)
        out = lcmg_result(x=_ptr(x), rho=_ptr(rho) if mo == 0 else None, eta=_ptr(eta) if mo == 0 else None,
                          iters=_ptr(its) if mo == 0 else None, status=_ptr(st) if mo == 0 else None,
                          history=_ptr(hist) if mo > 0 else None)
        code = fn(C.byref(out))
        if code == LCMG_ERR_NOT_READY:
            return None
        del self._reqs[ticket]
        if code != LCMG_OK:
            raise LcmgError(code, lib().lcmg_server_last_error().decode())
        r = dict(state=out.state, t_submit=out.t_submit, t_admit=out.t_admit, t_done=out.t_done,
                 n_solves=out.n_solves, n_converged=out.n_converged, x=x)
        if out.state != LCMG_OK:
            r["error"] = lib().lcmg_server_last_error().decode()
        if mo == 0:
            r.update(rho=rho, eta=eta, iters=its, status=st)
        else:
            r.update(history=list(hist[:out.n_outer]), n_outer=out.n_outer)
        return r

    def poll(self, ticket):
        return self._result(ticket, lambda o: lib().lcmg_server_poll(self.h, ticket, o))

    def wait(self, ticket, timeout=0.0):
        return self._result(ticket, lambda o: lib().lcmg_server_wait(self.h, ticket, timeout, o))

    def cancel(self, ticket):
        code = lib().lcmg_server_cancel(self.h, ticket)
        return code

    def stats(self):
        s = lcmg_server_stats()
        _scheck(lib().lcmg_server_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def footprint(self, problem, n_cols):
        v = C.c_size_t()
        _scheck(lib().lcmg_server_footprint(self.h, problem, n_cols, C.byref(v)))
        return v.value

    def close(self):
        if self.h:
            lib().lcmg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
