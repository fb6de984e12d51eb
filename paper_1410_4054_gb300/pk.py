"""Thin ctypes binding of the pk C ABI (include/pk.h): argument marshalling only.

Every numerical step runs in the CUDA library ``_build/libpk.so``; there is no CPU fallback.
``lib()`` loads it on first use (building it first if it is missing or stale); if it cannot
be built or loaded, that call and every call through it raise.  Vectors may be torch
CUDA tensors (passed by device pointer, on the current torch stream unless ``stream`` is
given) or numpy arrays / torch CPU tensors (host pointers: the library copies them in and out
inside the call).
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

from . import build as _build

PK_OK, PK_ERR_ARG, PK_ERR_CUDA, PK_ERR_OOM, PK_NOT_CONVERGED, PK_BREAKDOWN, PK_NOT_SPD, \
    PK_ERR_NAN, PK_TIMEOUT = range(9)
STATUS_NAMES = ["PK_OK", "PK_ERR_ARG", "PK_ERR_CUDA", "PK_ERR_OOM", "PK_NOT_CONVERGED",
                "PK_BREAKDOWN", "PK_NOT_SPD", "PK_ERR_NAN", "PK_TIMEOUT"]
VARIANTS = {"pipelined": 0, "classical": 1, "split": 2}
PRECISIONS = {"fp64": 0, "mixed": 1}
LOOPS = {"graph": 0, "host": 1, "persistent": 2, "auto": 3, "resident": 4}
PERSISTENT_AUTO_N = 65536  # PK_PERSISTENT_AUTO_N
PERSISTENT_AUTO_NNZ = 393216  # PK_PERSISTENT_AUTO_NNZ
PERSISTENT_BICGSTAB_AUTO_N = 32768  # PK_PERSISTENT_BICGSTAB_AUTO_N
PERSISTENT_BICGSTAB_AUTO_NNZ = 262144  # PK_PERSISTENT_BICGSTAB_AUTO_NNZ
PERSISTENT_GMRES_AUTO_N = 32768  # PK_PERSISTENT_GMRES_AUTO_N
PERSISTENT_GMRES_AUTO_NNZ = 262144  # PK_PERSISTENT_GMRES_AUTO_NNZ
FLAG_TIMING = 1
FLAG_TRUE_RES = 2
FLAG_NO_TMA = 4
FLAG_AUTOTUNE = 8
FLAG_SELL = 16
FLAG_CGS2 = 32
FLAG_TEST_STALL = 64
FLAG_GM_SHIFT = 128
SLOTS = ["spmv_dots", "update", "multidot", "ortho", "spmv", "blas1", "other", "resident"]
MAX_SLOTS = 8


class Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int32), ("restart", C.c_int32),
                ("variant", C.c_int32), ("precision", C.c_int32), ("loop", C.c_int32),
                ("check_every", C.c_int32), ("flags", C.c_uint32), ("trace_cap", C.c_int32),
                ("trace", C.c_void_p), ("precond", C.c_int32), ("lanes", C.c_int32),
                ("wait_ns", C.c_int64)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("cycles", C.c_int32),
                ("launches", C.c_int32), ("rel_res_est", C.c_double),
                ("rel_res_true", C.c_double), ("solve_ms", C.c_double),
                ("kernel_ms", C.c_double * MAX_SLOTS), ("kernel_count", C.c_int32 * MAX_SLOTS)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_min", C.c_int32),
                ("row_max", C.c_int32), ("row_mean", C.c_double), ("grid", C.c_int32),
                ("block", C.c_int32), ("kernel", C.c_int32), ("values_fp32_exact", C.c_int32),
                ("tiles_thread", C.c_int32), ("tiles_long", C.c_int32),
                ("tiles_group", C.c_int32), ("row_hist", C.c_int64 * 7)]


EXPORTS = {
    # name: (restype, argtypes)
    "pk_csr_create": (C.c_int, [C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "pk_csr_destroy": (C.c_int, [C.c_void_p]),
    "pk_csr_stats_get": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "pk_spmv": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pk_spmv_dot": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                              C.c_void_p]),
    "pk_cg_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Opts),
                              C.POINTER(Info), C.c_void_p]),
    "pk_spmv_dot_noalloc": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p]),
    "pk_bicgstab_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Opts),
                                    C.POINTER(Info), C.c_void_p]),
    "pk_gmres_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Opts),
                                 C.POINTER(Info), C.c_void_p]),
    "pk_gmres_cycle_factors": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pk_batched_solve": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Opts),
                                   C.c_void_p, C.c_void_p]),
    "pk_batched_last_config": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "pk_batched_last_lanes": (C.c_int, [C.POINTER(C.c_int32)]),
    "pk_csr_plan": (C.c_int, [C.c_int64, C.c_int64, C.c_void_p, C.c_int32, C.POINTER(Stats)]),
    "pk_residual_norm2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pk_conv3d_fwd": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "pk_conv3d_wgrad_scratch_floats": (C.c_int64, [C.c_int32, C.c_int32, C.c_int32]),
    "pk_conv3d_wgrad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    "pk_conv3d_flip": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "pk_conv3d_check": (C.c_int, [C.c_void_p]),
    "pk_warmstart_scratch_doubles": (C.c_int64, []),
    "pk_warmstart_input": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p]),
    "pk_warmstart_loss": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pk_warmstart_apply": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p]),
    "pk_warmstart_apply_energy": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "pk_warmstart_relax": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                     C.c_void_p]),
    "pk_warmstart_loss_swept": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_double, C.c_int32, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p]),
    "pk_adam_step": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_float,
                               C.c_float, C.c_float, C.c_float, C.c_int32, C.c_void_p, C.c_void_p]),
    "pk_status_string": (C.c_char_p, [C.c_int]),
    "pk_last_error": (C.c_char_p, []),
    "pk_version": (C.c_int32, []),
}

_lib = None


def lib_path() -> Path:
    return _build.LIB


def lib():
    """Load libpk.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(str(path))
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PkError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().pk_last_error().decode()
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 9 else status} {msg}")
        self.status = status


def _check(st: int, where: str, allow=(PK_OK,)):
    if st not in allow:
        raise PkError(st, where)
    return st


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:  # pragma: no cover
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(v):
    """Device or host pointer of a float64 torch tensor / numpy array."""
    if v is None:
        return C.c_void_p(0)
    if isinstance(v, np.ndarray):
        assert v.flags["C_CONTIGUOUS"], "array must be contiguous"
        return C.c_void_p(v.ctypes.data)
    assert v.is_contiguous(), "tensor must be contiguous"
    return C.c_void_p(v.data_ptr())


class CSRMatrix:
    """pk_csr handle: a library-owned device copy of a CSR matrix plus its schedule."""

    def __init__(self, row_ptr, col, val, n=None, stream=None):
        import torch

        if isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda:
            on_device = 1
            rp, ci, va = row_ptr.contiguous(), col.contiguous(), val.contiguous()
        else:
            on_device = 0
            rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
            ci = np.ascontiguousarray(col, dtype=np.int32)
            va = np.ascontiguousarray(val, dtype=np.float64)
        self._keep = (rp, ci, va)
        n = int(len(rp) - 1) if n is None else int(n)
        nnz = int(len(ci))
        h = C.c_void_p()
        _check(lib().pk_csr_create(n, nnz, _ptr(rp), _ptr(ci), _ptr(va), on_device,
                                   _stream_ptr(stream), C.byref(h)), "pk_csr_create")
        self.handle = h
        self.n, self.nnz = n, nnz
        self._keep = None

    @classmethod
    def from_workload(cls, a, stream=None):
        return cls(a.row_ptr, a.col, a.val, n=a.n, stream=stream)

    def stats(self) -> dict:
        s = Stats()
        _check(lib().pk_csr_stats_get(self.handle, C.byref(s)), "pk_csr_stats_get")
        d = {k: getattr(s, k) for k, _ in Stats._fields_}
        d["row_hist"] = list(d["row_hist"])  # rows with 0-8, 9-16, 17-32, 33-64, 65-256, 257-4096, > 4096 nonzeros
        return d

    def close(self):
        if getattr(self, "handle", None):
            lib().pk_csr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PRECONDS = {"none": 0, "jacobi": 1}


def make_opts(tol=1e-8, maxit=1000, restart=30, variant="pipelined", precision="fp64",
              loop="auto", check_every=0, flags=0, trace=None, precond="none", lanes=0,
              wait_ns=0) -> Opts:
    o = Opts()
    o.precond = PRECONDS[precond] if isinstance(precond, str) else int(precond)
    o.lanes = int(lanes)
    o.wait_ns = int(wait_ns)
    o.tol = tol
    o.maxit = maxit
    o.restart = restart
    o.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.loop = LOOPS[loop] if isinstance(loop, str) else int(loop)
    o.check_every = check_every
    o.flags = flags
    if trace is not None:
        assert trace.dim() == 2 and trace.shape[1] == 4 and trace.dtype.is_floating_point
        o.trace_cap = trace.shape[0]
        o.trace = trace.data_ptr()
    else:
        o.trace_cap = 0
        o.trace = None
    return o


def info_dict(info: Info) -> dict:
    d = {k: getattr(info, k) for k in ("iters", "status", "cycles", "launches", "rel_res_est",
                                       "rel_res_true", "solve_ms")}
    d["status_name"] = STATUS_NAMES[info.status] if 0 <= info.status < 9 else str(info.status)
    d["kernel_ms"] = {SLOTS[k]: info.kernel_ms[k] for k in range(len(SLOTS)) if info.kernel_count[k]}
    d["kernel_count"] = {SLOTS[k]: info.kernel_count[k] for k in range(len(SLOTS)) if info.kernel_count[k]}
    return d


_SOLVER_OK = (PK_OK, PK_NOT_CONVERGED, PK_BREAKDOWN, PK_NOT_SPD, PK_ERR_NAN)


def cg_solve(A: CSRMatrix, b, x, stream=None, **kw) -> dict:
    """pk_cg_solve: x (in: x0, out: solution)."""
    o = make_opts(**kw)
    info = Info()
    st = lib().pk_cg_solve(A.handle, _ptr(b), _ptr(x), C.byref(o), C.byref(info), _stream_ptr(stream))
    _check(st, "pk_cg_solve", _SOLVER_OK)
    return info_dict(info)


def bicgstab_solve(A: CSRMatrix, b, x, stream=None, **kw) -> dict:
    """pk_bicgstab_solve: x (in: x0, out: solution)."""
    o = make_opts(**kw)
    info = Info()
    st = lib().pk_bicgstab_solve(A.handle, _ptr(b), _ptr(x), C.byref(o), C.byref(info),
                                 _stream_ptr(stream))
    _check(st, "pk_bicgstab_solve", _SOLVER_OK)
    return info_dict(info)


def gmres_solve(A: CSRMatrix, b, x, stream=None, **kw) -> dict:
    """pk_gmres_solve (restart length = kw['restart']): x (in: x0, out: solution)."""
    o = make_opts(**kw)
    info = Info()
    st = lib().pk_gmres_solve(A.handle, _ptr(b), _ptr(x), C.byref(o), C.byref(info),
                              _stream_ptr(stream))
    _check(st, "pk_gmres_solve", _SOLVER_OK)
    return info_dict(info)


def gmres_cycle_factors(A: CSRMatrix, m: int, stream=None):
    """pk_gmres_cycle_factors: (R, xi) of the last GMRES cycle on A, R[j-1, i-1] = R_{j,i}."""
    R = np.zeros((m, m))
    xi = np.zeros(m)
    _check(lib().pk_gmres_cycle_factors(A.handle, int(m), _ptr(R), _ptr(xi), _stream_ptr(stream)),
           "pk_gmres_cycle_factors")
    return R, xi


def batched_solve(As, bs, xs, stream=None, **kw) -> list:
    """pk_batched_solve over lists of CSRMatrix handles and device tensors b[k], x[k]."""
    nsys = len(As)
    o = make_opts(**kw)
    ha = (C.c_void_p * nsys)(*[A.handle.value for A in As])
    hb = (C.c_void_p * nsys)(*[b.data_ptr() for b in bs])
    hx = (C.c_void_p * nsys)(*[x.data_ptr() for x in xs])
    infos = (Info * nsys)()
    st = lib().pk_batched_solve(nsys, ha, hb, hx, C.byref(o), infos, _stream_ptr(stream))
    _check(st, "pk_batched_solve", _SOLVER_OK)
    return [info_dict(infos[k]) for k in range(nsys)]


def csr_plan(row_ptr, sms=152) -> dict:
    """pk_csr_plan: the statistics and tile schedule pk_csr_create would choose, computed on
    the host (no GPU needed)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    s = Stats()
    _check(lib().pk_csr_plan(len(rp) - 1, int(rp[-1]) if len(rp) else 0, _ptr(rp), int(sms), C.byref(s)),
           "pk_csr_plan")
    d = {k: getattr(s, k) for k, _ in Stats._fields_}
    d["row_hist"] = list(d["row_hist"])
    return d


def batched_last_lanes() -> int:
    """Lanes per row of the last pk_batched_solve call (-1: the tile engine, -2: the cluster
    engine)."""
    v = C.c_int32()
    _check(lib().pk_batched_last_lanes(C.byref(v)), "pk_batched_last_lanes")
    return v.value


def batched_last_config() -> tuple:
    b, p = C.c_int32(), C.c_int32()
    _check(lib().pk_batched_last_config(C.byref(b), C.byref(p)), "pk_batched_last_config")
    return b.value, p.value


def spmv(A: CSRMatrix, x, y, stream=None):
    _check(lib().pk_spmv(A.handle, _ptr(x), _ptr(y), _stream_ptr(stream)), "pk_spmv")


def spmv_dot(A: CSRMatrix, p, q, result, fused=True, stream=None, sell=False):
    """pk_spmv_dot: q = A p, result[0] = <p, q>; fused (one launch) or not; sell: the fused
    kernel on the SELL-C-sigma copy."""
    mode = 2 if sell else (1 if fused else 0)
    _check(lib().pk_spmv_dot(A.handle, _ptr(p), _ptr(q), _ptr(result), mode, _stream_ptr(stream)),
           "pk_spmv_dot")


def status_string(s: int) -> str:
    return lib().pk_status_string(s).decode()


def version() -> int:
    return lib().pk_version()


NOALLOC_MAX_N = 16777216


def spmv_dot_noalloc(n, row_ptr, col, val, p, q, result, stream=None):
    """pk_spmv_dot_noalloc: q = A p, result = <p, q> from device CSR arrays, no allocation."""
    _check(lib().pk_spmv_dot_noalloc(int(n), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(p), _ptr(q),
                                     _ptr(result), _stream_ptr(stream)), "pk_spmv_dot_noalloc")


def residual_norm2(A: CSRMatrix, b, x, out2, stream=None):
    """out2[0] = ||b - A x||^2 (device tensors)."""
    _check(lib().pk_residual_norm2(A.handle, _ptr(b), _ptr(x), _ptr(out2), _stream_ptr(stream)),
           "pk_residual_norm2")


def conv3d_check(stream=None):
    """Raises PkError(PK_TIMEOUT) if a tensor-core convolution timed out since the last check."""
    _check(lib().pk_conv3d_check(_stream_ptr(stream)), "pk_conv3d_check")


def conv3d_fwd(X, Wt, bias, Y, dims, relu=True, out_f32=False, mask=None, stream=None):
    D, H, W = dims
    _check(lib().pk_conv3d_fwd(_ptr(X), _ptr(Wt), _ptr(bias), _ptr(Y), D, H, W, int(relu),
                               int(out_f32), _ptr(mask), _stream_ptr(stream)), "pk_conv3d_fwd")


def conv3d_wgrad_scratch_floats(dims) -> int:
    return int(lib().pk_conv3d_wgrad_scratch_floats(*dims))


def conv3d_wgrad(A, G, scratch, dW, db, dims, stream=None):
    D, H, W = dims
    _check(lib().pk_conv3d_wgrad(_ptr(A), _ptr(G), _ptr(scratch), _ptr(dW), _ptr(db), D, H, W,
                                 _stream_ptr(stream)), "pk_conv3d_wgrad")


def conv3d_flip(W, Wf, stream=None):
    _check(lib().pk_conv3d_flip(_ptr(W), _ptr(Wf), _stream_ptr(stream)), "pk_conv3d_flip")


def warmstart_scratch_doubles() -> int:
    return int(lib().pk_warmstart_scratch_doubles())


def warmstart_input(A: CSRMatrix, xm1, xm2, b, X16, scales, scratch, stream=None):
    _check(lib().pk_warmstart_input(A.handle, _ptr(xm1), _ptr(xm2), _ptr(b), _ptr(X16), _ptr(scales),
                                    _ptr(scratch), _stream_ptr(stream)), "pk_warmstart_input")


def warmstart_loss(n, out, xt, xm1, xm2, scales, G, loss, scratch, stream=None):
    _check(lib().pk_warmstart_loss(int(n), _ptr(out), _ptr(xt), _ptr(xm1), _ptr(xm2), _ptr(scales),
                                   _ptr(G), _ptr(loss), _ptr(scratch), _stream_ptr(stream)),
           "pk_warmstart_loss")


def warmstart_apply(n, out, xm1, xm2, scales, xhat, stream=None):
    """x_hat = 2 x_{t-1} - x_{t-2} + s out (out None: the extrapolation alone)."""
    _check(lib().pk_warmstart_apply(int(n), _ptr(out), _ptr(xm1), _ptr(xm2), _ptr(scales), _ptr(xhat),
                                    _stream_ptr(stream)), "pk_warmstart_apply")


def warmstart_apply_energy(A: CSRMatrix, out, xm1, xm2, b, scales, xhat, gamma, scratch, stream=None):
    """x_hat = e + gamma s0 out with the A-norm-optimal gamma (written to gamma[0])."""
    _check(lib().pk_warmstart_apply_energy(A.handle, _ptr(out), _ptr(xm1), _ptr(xm2), _ptr(b), _ptr(scales),
                                           _ptr(xhat), _ptr(gamma), _ptr(scratch), _stream_ptr(stream)),
           "pk_warmstart_apply_energy")


def warmstart_relax(A: CSRMatrix, b, x, omega, xout, stream=None):
    """xout = x + omega (b - A x) / diag(A): one damped Jacobi sweep (xout must not be x)."""
    _check(lib().pk_warmstart_relax(A.handle, _ptr(b), _ptr(x), float(omega), _ptr(xout), _stream_ptr(stream)),
           "pk_warmstart_relax")


def warmstart_loss_swept(A: CSRMatrix, out, xt, xm1, xm2, scales, omega, sweeps, G, loss, work, scratch,
                         stream=None):
    """Loss and output gradient of the guess after `sweeps` Jacobi sweeps (A symmetric)."""
    _check(lib().pk_warmstart_loss_swept(A.handle, _ptr(out), _ptr(xt), _ptr(xm1), _ptr(xm2), _ptr(scales),
                                         float(omega), int(sweeps), _ptr(G), _ptr(loss), _ptr(work),
                                         _ptr(scratch), _stream_ptr(stream)), "pk_warmstart_loss_swept")


def adam_step(p, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, p_bf16=None, stream=None):
    _check(lib().pk_adam_step(p.numel(), _ptr(p), _ptr(grad), _ptr(m), _ptr(v), lr, beta1, beta2, eps,
                              int(step), _ptr(p_bf16), _stream_ptr(stream)), "pk_adam_step")
