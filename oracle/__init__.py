"""CPU oracle for the pipelined Krylov solvers (Rupp et al., arXiv:1410.4054).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this package.  The
product path (the CUDA library and its Python binding) never does, and the two share no
code: the arithmetic lives in ``pk_oracle.c`` (plain sequential FP64 C, compiled with
``-ffp-contract=off``) and in ``conv3d.py`` (numpy FP64); this module only marshals numpy
arrays into it.

Every function returns a plain dict with the solution, iteration count, status and the
per-iteration scalar traces of the algorithm it follows.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

# status codes of the oracle (same meaning as the library's, defined independently)
OK, ERR_ARG, ERR_OOM, NOT_CONVERGED, BREAKDOWN, NOT_SPD, NAN = 0, 1, 3, 4, 5, 6, 7

_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_dp = C.c_void_p  # nullable double*


def lib():
    global _lib
    if _lib is None:
        # PK_ORACLE_LIB lets the mutation test load a deliberately broken build of the oracle
        path = os.environ.get("PK_ORACLE_LIB") or _build.build()
        L = C.CDLL(str(path))
        L.orc_spmv.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.orc_spmv.restype = None
        L.orc_dot.argtypes = [C.c_int32, _f64p, _f64p]
        L.orc_dot.restype = C.c_double
        common = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, C.c_double, C.c_int32, C.c_int32]
        for name in ("orc_cg_classical", "orc_cg_pipelined"):
            f = getattr(L, name)
            f.argtypes = common + [_dp, _dp, _dp, C.POINTER(C.c_int32)]
            f.restype = C.c_int
        L.orc_pcg_jacobi.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, C.c_double, C.c_int32,
                                     C.c_int32, C.c_int32, _dp, _dp, _dp, C.POINTER(C.c_int32)]
        L.orc_pcg_jacobi.restype = C.c_int
        L.orc_bicgstab_classical.argtypes = common + [_dp, _dp, _dp, _dp, C.POINTER(C.c_int32)]
        L.orc_bicgstab_classical.restype = C.c_int
        L.orc_bicgstab_pipelined.argtypes = common + [_dp, _dp, _dp, _dp, _dp, C.POINTER(C.c_int32)]
        L.orc_bicgstab_pipelined.restype = C.c_int
        L.orc_gmres.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, C.c_double,
                                C.c_int32, C.c_int32, C.c_int32, C.c_int32, _dp, _dp, _dp, _dp,
                                C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.orc_gmres.restype = C.c_int
        L.orc_gmres_cgs2.argtypes = L.orc_gmres.argtypes + [_dp]
        L.orc_gmres_cgs2.restype = C.c_int
        L.orc_gmres_shift3.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, C.c_double,
                                       C.c_int32, C.c_int32, C.c_int32, _dp, _dp, _dp, _dp, _dp,
                                       C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.orc_gmres_shift3.restype = C.c_int
        L.orc_jacobi_right_begin.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
        L.orc_jacobi_right_begin.restype = C.c_int
        L.orc_jacobi_right_end.argtypes = [C.c_int32, _f64p, _f64p]
        L.orc_jacobi_right_end.restype = None
        _lib = L
    return _lib


def _csr(a):
    return (int(a.n), np.ascontiguousarray(a.row_ptr, dtype=np.int32),
            np.ascontiguousarray(a.col, dtype=np.int32), np.ascontiguousarray(a.val, dtype=np.float64))


def _ptr(arr):
    return arr.ctypes.data_as(C.c_void_p)


def spmv(a, x):
    n, rp, ci, va = _csr(a)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n)
    lib().orc_spmv(n, rp, ci, va, x, y)
    return y


def dot(x, y):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return lib().orc_dot(x.size, x, y)


def cg(a, b, x0=None, tol=1e-8, maxit=1000, variant="pipelined", cap=None):
    """Algorithm 1 (variant='classical') or Algorithm 2 (variant='pipelined')."""
    n, rp, ci, va = _csr(a)
    cap = maxit + 1 if cap is None else cap
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    tr = {k: np.full(cap, np.nan) for k in ("alpha", "beta", "res2")}
    it = C.c_int32(0)
    f = lib().orc_cg_pipelined if variant == "pipelined" else lib().orc_cg_classical
    st = f(n, rp, ci, va, b, x, tol, maxit, cap, _ptr(tr["alpha"]), _ptr(tr["beta"]),
           _ptr(tr["res2"]), C.byref(it))
    return dict(x=x, iters=it.value, status=st, **tr)


def pcg_jacobi(a, b, x0=None, tol=1e-8, maxit=1000, variant="pipelined", cap=None):
    """CG with the Jacobi preconditioner diag(A): standard (variant='classical') or in the
    pipelined structure of Algorithm 2 (variant='pipelined')."""
    n, rp, ci, va = _csr(a)
    cap = maxit + 1 if cap is None else cap
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    tr = {k: np.full(cap, np.nan) for k in ("alpha", "beta", "res2")}
    it = C.c_int32(0)
    st = lib().orc_pcg_jacobi(n, rp, ci, va, b, x, tol, maxit, 1 if variant == "pipelined" else 0, cap,
                              _ptr(tr["alpha"]), _ptr(tr["beta"]), _ptr(tr["res2"]), C.byref(it))
    return dict(x=x, iters=it.value, status=st, **tr)


def _right_jacobi(n, rp, ci, va, x, precond):
    """precond='jacobi': the values of A M^-1 and M^-1 (M = diag(A)), x <- M x; else as given."""
    if precond == "none":
        return va, None
    if precond != "jacobi":
        raise ValueError(f"precond {precond!r}")
    va_r, dinv = np.empty_like(va), np.empty(n)
    if lib().orc_jacobi_right_begin(n, rp, ci, va, x, va_r, dinv) != OK:
        raise ValueError("the Jacobi preconditioner needs a nonzero finite diagonal")
    return va_r, dinv


def bicgstab(a, b, x0=None, tol=1e-8, maxit=1000, variant="pipelined", cap=None, precond="none"):
    """Algorithm 3 (variant='classical') or Algorithm 4 (variant='pipelined');
    precond='jacobi': right-preconditioned with M = diag(A) (run on A M^-1, x = M^-1 y)."""
    n, rp, ci, va = _csr(a)
    cap = maxit + 1 if cap is None else cap
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    va, dinv = _right_jacobi(n, rp, ci, va, x, precond)
    tr = {k: np.full(cap, np.nan) for k in ("alpha", "beta", "omega", "res2", "res2_est")}
    it = C.c_int32(0)
    if variant == "pipelined":
        st = lib().orc_bicgstab_pipelined(n, rp, ci, va, b, x, tol, maxit, cap, _ptr(tr["alpha"]),
                                          _ptr(tr["beta"]), _ptr(tr["omega"]), _ptr(tr["res2"]),
                                          _ptr(tr["res2_est"]), C.byref(it))
    else:
        st = lib().orc_bicgstab_classical(n, rp, ci, va, b, x, tol, maxit, cap, _ptr(tr["alpha"]),
                                          _ptr(tr["beta"]), _ptr(tr["omega"]), _ptr(tr["res2"]),
                                          C.byref(it))
    if dinv is not None:
        lib().orc_jacobi_right_end(n, dinv, x)
    return dict(x=x, iters=it.value, status=st, **tr)


def gmres(a, b, x0=None, tol=1e-8, maxit=1000, m=30, variant="pipelined", cap=None, precond="none",
          cgs2=False, shift3=False):
    """Algorithm 6 (variant='pipelined') or Algorithm 5 (variant='classical'), restarted;
    precond='jacobi': right-preconditioned with M = diag(A) (run on A M^-1, x = M^-1 y);
    cgs2: Gram-Schmidt applied twice per step; shift3: the shift-invariant three-kernel form
    of the pipelined method (Sec. 3.3), with the per-step shifts in 'sigma'."""
    n, rp, ci, va = _csr(a)
    cap = maxit + 2 if cap is None else cap
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    va, dinv = _right_jacobi(n, rp, ci, va, x, precond)
    R = np.zeros((m, m))
    xi = np.zeros(m)
    est = np.full(cap, np.nan)
    res = np.full(cap, np.nan)
    it, cyc = C.c_int32(0), C.c_int32(0)
    if shift3:
        if variant != "pipelined" or cgs2:
            raise ValueError("the three-kernel form is a form of the pipelined method with one Gram-Schmidt pass")
        sigma = np.full(cap, np.nan)
        st = lib().orc_gmres_shift3(n, rp, ci, va, b, x, tol, maxit, m, cap, _ptr(R), _ptr(xi), _ptr(est),
                                    _ptr(res), _ptr(sigma), C.byref(it), C.byref(cyc))
        if dinv is not None:
            lib().orc_jacobi_right_end(n, dinv, x)
        return dict(x=x, iters=it.value, cycles=cyc.value, status=st, R=R, xi=xi, est=est, res=res,
                    sigma=sigma)
    args = (n, rp, ci, va, b, x, tol, maxit, m, 1 if variant == "pipelined" else 0,
            cap, _ptr(R), _ptr(xi), _ptr(est), _ptr(res), C.byref(it), C.byref(cyc))
    V = None
    if cgs2:
        V = np.full((m + 1, n), np.nan)
        st = lib().orc_gmres_cgs2(*args, _ptr(V))
    else:
        st = lib().orc_gmres(*args)
    if dinv is not None:
        lib().orc_jacobi_right_end(n, dinv, x)
    out = dict(x=x, iters=it.value, cycles=cyc.value, status=st, R=R, xi=xi, est=est, res=res)
    if V is not None:
        out["V"] = V   # first cycle's basis v_0 .. v_k (rows beyond k: NaN)
    return out


_omp = None


def omp_lib():
    """The OpenMP timing copy of the pipelined CG oracle (libpk_oracle_omp.so), or None when
    the compiler has no OpenMP.  Used only for the CPU baseline's multi-threaded leg."""
    global _omp
    if _omp is None:
        try:
            path = _build.build_omp()
        except Exception:  # noqa: BLE001 - no OpenMP on this host: single-threaded leg only
            return None
        L = C.CDLL(str(path))
        L.orc_omp_threads.argtypes = []
        L.orc_omp_threads.restype = C.c_int32
        L.orc_omp_set_threads.argtypes = [C.c_int32]
        L.orc_omp_set_threads.restype = None
        L.orc_cg_pipelined_omp.argtypes = [C.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, C.c_double,
                                           C.c_int32, C.POINTER(C.c_int32)]
        L.orc_cg_pipelined_omp.restype = C.c_int
        _omp = L
    return _omp


def cg_omp(a, b, x0=None, tol=1e-8, maxit=1000, threads=None):
    """Algorithm 2 with every row loop split statically over `threads` OpenMP threads (default:
    the cores this process may run on).  Timing only: the parity oracle is cg()."""
    L = omp_lib()
    if L is None:
        raise RuntimeError("the OpenMP oracle is not available (gcc without -fopenmp)")
    n, rp, ci, va = _csr(a)
    threads = threads or len(os.sched_getaffinity(0))
    L.orc_omp_set_threads(int(threads))
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it = C.c_int32(0)
    st = L.orc_cg_pipelined_omp(n, rp, ci, va, b, x, tol, maxit, C.byref(it))
    return dict(x=x, iters=it.value, status=st, threads=int(L.orc_omp_threads()))
