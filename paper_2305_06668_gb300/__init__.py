"""GB300 LOBPCG eigensolver: thin Python binding of the C ABI in include/lobpcg.h.

The binding only marshals arguments: every step of the method runs in the CUDA kernels
of ``_build/liblobpcg.so``.  PyTorch supplies device memory and the current stream.
There is no CPU fallback: without the compiled library every call raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import pathlib

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_LIB_PATH = _HERE / "_build" / "liblobpcg.so"
_lib = None

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, EBREAKDOWN = range(6)
CSR, DENSE = 0, 1
PREC_NONE, PREC_DIAG, PREC_LEARNED, PREC_TRIDIAG = 0, 1, 2, 3
FP64, MIXED = 0, 1
PHASES = ("spmm", "rr_gram", "rr_eig", "update_lock", "precond", "ortho")
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "EBREAKDOWN"}


class LobpcgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _Matrix(C.Structure):
    _fields_ = [("fmt", C.c_int), ("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p), ("dense", C.c_void_p), ("ld", C.c_int64),
                ("diag", C.c_void_p)]


class _Options(C.Structure):
    _fields_ = [("extra", C.c_int), ("maxiter", C.c_int), ("tol_kind", C.c_int), ("precond", C.c_int),
                ("precision", C.c_int), ("tau_ortho", C.c_double), ("ortho_cap", C.c_int),
                ("ortho2_cap", C.c_int), ("seed", C.c_uint64), ("mlp_weights", C.c_void_p), ("profile", C.c_int),
                ("mixed_switch", C.c_double), ("autotune", C.c_int), ("ortho_trim", C.c_int),
                ("df_products", C.c_int), ("tc_gram", C.c_int), ("precond_floor", C.c_double)]


class _Info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("fp64_iterations", C.c_int), ("converged", C.c_int),
                ("cholqr_passes_max", C.c_int), ("ortho_passes_max", C.c_int), ("shifts", C.c_int),
                ("svqb", C.c_int), ("cap_hits", C.c_int), ("spmm_columns", C.c_int64),
                ("seconds", C.c_double), ("phase_seconds", C.c_double * 6), ("kernel_launches", C.c_int64),
                ("spmm_launches", C.c_int64), ("precond_fallback", C.c_int),
                ("phase_seconds_fp64", C.c_double * 6), ("spmm_launches_fp64", C.c_int64),
                ("spmm_columns_fp64", C.c_int64), ("update_fp64_seconds", C.c_double),
                ("update_fp64_flops", C.c_double), ("update_fp64_launches", C.c_int64),
                ("spmm_variant_fp32", C.c_int), ("spmm_variant_fp64", C.c_int), ("w_dropped", C.c_int),
                ("p_dropped", C.c_int), ("ortho_grams", C.c_int), ("skipped_recheck", C.c_int),
                ("skipped_test", C.c_int), ("df_products", C.c_int), ("rr_gram32_bytes", C.c_double),
                ("rr_gram32_count", C.c_int64)]


def library_path() -> pathlib.Path:
    return _LIB_PATH


def lib():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise RuntimeError(f"CUDA library not built: {_LIB_PATH} is missing (run __graft_entry__.build())")
        L = C.CDLL(str(_LIB_PATH))
        for name in ("lobpcg_options_default", "lobpcg_create", "lobpcg_solve", "lobpcg_spmm_csr_f64",
                     "lobpcg_spmm_dense_f64", "lobpcg_gram_f64", "lobpcg_syev_f64", "lobpcg_ortho_f64",
                     "lobpcg_ortho_against_f64", "lobpcg_gram_f64_noalloc", "lobpcg_mlp_forward",
                     "lobpcg_mlp_backward", "lobpcg_mlp_loss", "lobpcg_mlp_adam", "lobpcg_precond_features",
                     "lobpcg_row_norms", "lobpcg_mlp_num_params", "lobpcg_solve_batched",
                     "lobpcg_spmm_csr_f32", "lobpcg_syev2_f64", "lobpcg_gram_f32", "lobpcg_update_f32",
                     "lobpcg_probe_fma_rate", "lobpcg_gram_f64_df", "lobpcg_update_f64_df",
                     "lobpcg_spmm_csr_f64_df", "lobpcg_gram_f32_tcgen05", "lobpcg_precond_tridiag",
                     "lobpcg_mixed_switch_replay"):
            getattr(L, name).restype = C.c_int
        L.lobpcg_last_error.restype = C.c_char_p
        L.lobpcg_last_error.argtypes = [C.c_void_p]
        L.lobpcg_destroy.restype = None
        L.lobpcg_destroy.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    """Names of the C entry points declared in include/lobpcg.h."""
    import re
    hdr = (_HERE.parent / "include" / "lobpcg.h").read_text()
    return re.findall(r"LOBPCG_API\s+[\w\s\*]+?\b(lobpcg_\w+)\s*\(", hdr)


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(0 if t is None else t.data_ptr())


def _check(status: int, ctx=None):
    if status != OK:
        msg = lib().lobpcg_last_error(ctx).decode()
        raise LobpcgError(status, msg)


def _need_cuda(t, dtype, name):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}")
    return t


@dataclasses.dataclass
class Result:
    status: int
    evals: np.ndarray
    evecs: object  # torch.Tensor (n, k), column-major storage
    resnorms: np.ndarray
    info: dict


class Solver:
    """Context for one symmetric matrix (lobpcg_create / lobpcg_solve / lobpcg_destroy).

    CSR: pass ``row_ptr`` (int64), ``col_idx`` (int32), ``val`` (float64) CUDA tensors.
    Dense: pass ``dense`` (float64, n x n, column-major storage or symmetric).
    ``diag`` (float64, n) is always required.  ``mass``: the matrix B of a generalised
    problem A x = lambda B x (Sec. 3.3), a dict with the same keys (row_ptr, col_idx, val or
    dense, and its diag).
    """

    def __init__(self, *, diag, row_ptr=None, col_idx=None, val=None, dense=None, extra: int = 0,
                 maxiter: int = 1000, tol_kind: int = 0, precond: int = PREC_DIAG, precision: int = FP64,
                 tau_ortho: float = 1e-14, ortho_cap: int = 6, ortho2_cap: int = 4, seed: int = 0,
                 mlp_weights=None, profile: bool = False, mixed_switch: float = 0.0, autotune: bool = False,
                 ortho_trim: bool = True, df_products: int = 0, tc_gram: bool = True, precond_floor: float = 0.0,
                 mass=None, stream=None):
        torch = _torch()
        L = lib()
        self._keep = [diag, row_ptr, col_idx, val, dense, mass]
        _need_cuda(diag, torch.float64, "diag")
        n = diag.numel()
        m = _Matrix()
        if dense is not None:
            _need_cuda(dense, torch.float64, "dense")
            m.fmt, m.n, m.dense, m.ld = DENSE, n, dense.data_ptr(), n
            if not (dense.is_contiguous() or dense.t().is_contiguous()):
                raise ValueError("dense must be contiguous (row- or column-major; A is symmetric)")
        else:
            _need_cuda(row_ptr, torch.int64, "row_ptr")
            _need_cuda(col_idx, torch.int32, "col_idx")
            _need_cuda(val, torch.float64, "val")
            m.fmt, m.n, m.nnz = CSR, n, val.numel()
            m.row_ptr, m.col_idx, m.val = row_ptr.data_ptr(), col_idx.data_ptr(), val.data_ptr()
        m.diag = diag.data_ptr()
        o = _Options()
        L.lobpcg_options_default(C.byref(o))
        o.extra, o.maxiter, o.tol_kind, o.precond, o.precision = extra, maxiter, tol_kind, precond, precision
        o.tau_ortho, o.ortho_cap, o.ortho2_cap, o.seed = tau_ortho, ortho_cap, ortho2_cap, seed
        o.profile = 1 if profile else 0
        o.mixed_switch = mixed_switch
        o.autotune = 1 if autotune else 0
        o.ortho_trim = 1 if ortho_trim else 0
        o.df_products = int(df_products)
        o.tc_gram = 1 if tc_gram else 0
        o.precond_floor = float(precond_floor)
        w = None
        if mlp_weights is not None:
            w = np.ascontiguousarray(mlp_weights, dtype=np.float32)
            o.mlp_weights = w.ctypes.data
        self.n, self.extra = n, extra
        self._stream_obj = stream if stream is not None else torch.cuda.current_stream()
        self._ctx = C.c_void_p()
        if mass is None:
            _check(L.lobpcg_create(C.byref(self._ctx), C.byref(m), C.byref(o), _stream(self._stream_obj)), None)
        else:
            mb = _Matrix()
            _need_cuda(mass["diag"], torch.float64, "mass diag")
            mb.n, mb.diag = mass["diag"].numel(), mass["diag"].data_ptr()
            if mass.get("dense") is not None:
                _need_cuda(mass["dense"], torch.float64, "mass dense")
                mb.fmt, mb.dense, mb.ld = DENSE, mass["dense"].data_ptr(), n
            else:
                for key, dt in (("row_ptr", torch.int64), ("col_idx", torch.int32), ("val", torch.float64)):
                    _need_cuda(mass[key], dt, "mass " + key)
                mb.fmt, mb.nnz = CSR, mass["val"].numel()
                mb.row_ptr, mb.col_idx, mb.val = (mass["row_ptr"].data_ptr(), mass["col_idx"].data_ptr(),
                                                  mass["val"].data_ptr())
            L.lobpcg_create_gen.restype = C.c_int
            _check(L.lobpcg_create_gen(C.byref(self._ctx), C.byref(m), C.byref(mb), C.byref(o),
                                       _stream(self._stream_obj)), None)

    def solve(self, k: int, tol: float = 1e-8, X0=None, raise_on_noconv: bool = False) -> Result:
        torch = _torch()
        m = k + self.extra
        if X0 is not None:
            _need_cuda(X0, torch.float64, "X0")
            if tuple(X0.shape) != (self.n, m):
                raise ValueError(f"X0 must be {self.n} x {m}")
            X0 = X0.t().contiguous().t()  # column-major storage
        evecs = torch.empty((k, self.n), dtype=torch.float64, device="cuda").t()
        evals = np.zeros(k)
        res = np.zeros(k)
        info = _Info()
        st = lib().lobpcg_solve(self._ctx, C.c_int(k), C.c_double(tol), _ptr(X0),
                                evals.ctypes.data_as(C.c_void_p), C.c_void_p(evecs.data_ptr()),
                                res.ctypes.data_as(C.c_void_p), C.byref(info))
        if st not in (OK, ENOCONV) or (raise_on_noconv and st == ENOCONV):
            _check(st, self._ctx)
        d = {f: getattr(info, f) for f, _ in _Info._fields_}
        d["phase_seconds"] = dict(zip(PHASES, list(info.phase_seconds)))
        d["phase_seconds_fp64"] = dict(zip(PHASES, list(info.phase_seconds_fp64)))
        return Result(st, evals, evecs, res, d)

    @property
    def handle(self):
        return self._ctx

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().lobpcg_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ building blocks
# Row-major blocks: a contiguous (n, p) torch tensor is exactly the layout of the C ABI.

def spmm_csr(row_ptr, col_idx, val, X, stream=None):
    torch = _torch()
    n, p = X.shape
    Y = torch.empty_like(X)
    _check(lib().lobpcg_spmm_csr_f64(C.c_int64(n), _ptr(row_ptr), _ptr(col_idx), _ptr(val), C.c_int(p),
                                     _ptr(X), C.c_int(X.stride(0)), _ptr(Y), C.c_int(Y.stride(0)), _stream(stream)))
    return Y


def spmm_csr_f32(row_ptr, col_idx, val, X, band=-1, stream=None):
    """FP32 product of the mixed form: Y = fp32(A) X for a float32 row-major block X whose
    leading dimension is a multiple of 4 (pad the columns if needed).  band: -1 automatic
    band / long-range split, >= 0 forced half-width, -2 unsplit.  Returns (Y, band used)."""
    torch = _torch()
    n, p = X.shape
    if X.dtype != torch.float32:
        raise TypeError("spmm_csr_f32: X must be float32")
    Y = torch.empty((n, X.stride(0)), dtype=X.dtype, device=X.device)[:, :p]
    used = C.c_int(0)
    _check(lib().lobpcg_spmm_csr_f32(C.c_int64(n), _ptr(row_ptr), _ptr(col_idx), _ptr(val),
                                     C.c_int64(val.numel()), C.c_int(p), _ptr(X), C.c_int(X.stride(0)), _ptr(Y),
                                     C.c_int(Y.stride(0)), C.c_int(band), C.byref(used), _stream(stream)))
    return Y, used.value


def mixed_switch_replay(rk, switch_tol: float = 0.0) -> int:
    """The FP32 iteration after which the mixed form would leave FP32 for the residual
    history rk (largest sought residual per iteration), or -1 (lobpcg_mixed_switch_replay)."""
    import numpy as np
    r = np.ascontiguousarray(rk, dtype=np.float64)
    out = C.c_int(0)
    _check(lib().lobpcg_mixed_switch_replay(r.ctypes.data_as(C.c_void_p) if r.size else None, C.c_int(r.size),
                                            C.c_double(switch_tol), C.byref(out)))
    return out.value


def precond_tridiag(dl, d, du, shift, R, stream=None):
    """W[:, j] = (T - shift[j] I)^{-1} R[:, j] for the tridiagonal T = (dl, d, du) (FP64 device
    tensors; R row-major n x p).  Returns W (n x p, float64)."""
    torch = _torch()
    n, p = R.shape
    W = torch.empty((n, p), dtype=torch.float64, device=R.device)
    _check(lib().lobpcg_precond_tridiag(C.c_int64(n), _ptr(dl) if n > 1 else None, _ptr(d),
                                        _ptr(du) if n > 1 else None, C.c_int(p), _ptr(shift), _ptr(R),
                                        C.c_int(R.stride(0)), _ptr(W), C.c_int(W.stride(0)), _stream(stream)))
    return W


def spmm_dense(A, X, stream=None):
    torch = _torch()
    n, p = X.shape
    Y = torch.empty_like(X)
    At = A if A.t().is_contiguous() else A.t().contiguous().t()  # column-major storage
    _check(lib().lobpcg_spmm_dense_f64(C.c_int64(n), _ptr(At), C.c_int64(n), C.c_int(p), _ptr(X),
                                       C.c_int(X.stride(0)), _ptr(Y), C.c_int(Y.stride(0)), _stream(stream)))
    return Y


def gram(X, Y, stream=None):
    """C = X^T Y for row-major blocks X (n x p), Y (n x q)."""
    torch = _torch()
    n, p = X.shape
    q = Y.shape[1]
    Cm = torch.empty((q, p), dtype=torch.float64, device=X.device)  # column-major p x q
    _check(lib().lobpcg_gram_f64(C.c_int64(n), C.c_int(p), _ptr(X), C.c_int(X.stride(0)), C.c_int(q), _ptr(Y),
                                 C.c_int(Y.stride(0)), _ptr(Cm), _stream(stream)))
    return Cm.t()


def gram_f32(X, Y, stream=None):
    """C = X^T Y (FP64 result) for float32 row-major blocks X (n x p), Y (n x q)."""
    torch = _torch()
    n, p = X.shape
    q = Y.shape[1]
    if X.dtype != torch.float32 or Y.dtype != torch.float32:
        raise TypeError("gram_f32: X and Y must be float32")
    Cm = torch.empty((q, p), dtype=torch.float64, device=X.device)
    _check(lib().lobpcg_gram_f32(C.c_int64(n), C.c_int(p), _ptr(X), C.c_int(X.stride(0)), C.c_int(q), _ptr(Y),
                                 C.c_int(Y.stride(0)), _ptr(Cm), _stream(stream)))
    return Cm.t()


def update_f32(V, U, q=None, alpha=1.0, AV=None, base=None, X=None, AX=None, lam=None, resnorm=False,
               stream=None):
    """X = base + alpha [V_0 ..] U and, with AV, AX = alpha [AV_0 ..] U (FP32 block update).

    V (and AV): a list of 1 to 3 float32 CUDA tensors (n x w_g views sharing one row
    stride); U: float64 CUDA (s x q) with s = sum of w_g.  base, X, AX: optional float32
    (n x q, X and AX sharing one row stride; X may be base or V[0] for an in-place update).
    With resnorm=True (AV and lam given, no base) also returns || AX_j - lam_j X_j ||_2.
    Returns X, or (X, AX), or (X, AX, resnorm).
    """
    torch = _torch()
    V = list(V)
    n = V[0].shape[0]
    ws = [int(v.shape[1]) for v in V]
    ld = int(V[0].stride(0))
    q = int(U.shape[1]) if q is None else int(q)
    if X is None:
        X = torch.empty((n, q), dtype=torch.float32, device=V[0].device)
    if AV is not None and AX is None:
        AX = torch.empty_like(X)
    Ucol = U if (U.stride(0) == 1 and U.stride(1) == U.shape[0]) else U.t().contiguous().t()  # column-major
    vp = (C.c_void_p * len(V))(*[v.data_ptr() for v in V])
    ap = (C.c_void_p * len(V))(*[a.data_ptr() for a in AV]) if AV is not None else None
    warr = (C.c_int * len(V))(*ws)
    rn = (C.c_double * q)() if resnorm else None
    _check(lib().lobpcg_update_f32(C.c_int64(n), C.c_int(len(V)), vp, ap, warr, C.c_int(ld), _ptr(Ucol),
                                   C.c_int(q), C.c_double(alpha), _ptr(base),
                                   C.c_int(base.stride(0) if base is not None else 0), _ptr(X), _ptr(AX),
                                   C.c_int(X.stride(0)), _ptr(lam), rn, _stream(stream)))
    if AV is None:
        return X
    if resnorm:
        return X, AX, np.array(rn[:])
    return X, AX


def probe_fma_rate(fp64: bool = True, stream=None) -> float:
    """Measured peak FMA rate of the current GPU in TFLOP/s (FP64 or FP32 pipes)."""
    out = C.c_double(0.0)
    _check(lib().lobpcg_probe_fma_rate(C.c_int(1 if fp64 else 0), C.byref(out), _stream(stream)))
    return out.value


def spmm_csr_df(row_ptr, col_idx, val, X, Y=None, stream=None):
    """Y = A X (CSR A, FP64 row-major X) in double-float arithmetic (the refinement's product)."""
    torch = _torch()
    n, p = X.shape
    if Y is None:
        Y = torch.empty_like(X)
    _check(lib().lobpcg_spmm_csr_f64_df(C.c_int64(n), _ptr(row_ptr), _ptr(col_idx), _ptr(val),
                                        C.c_int64(val.numel()), C.c_int(p), _ptr(X), C.c_int(X.stride(0)), _ptr(Y),
                                        C.c_int(Y.stride(0)), _stream(stream)))
    return Y


def gram_f32_tcgen05(X, Y, stream=None):
    """C = X^T Y of FP32 row-major CUDA blocks (one aligned row stride) on the tcgen05 tensor
    cores (3xTF32), FP64 result."""
    torch = _torch()
    n, p = X.shape
    q = Y.shape[1]
    Cm = torch.empty((q, p), dtype=torch.float64, device=X.device)
    _check(lib().lobpcg_gram_f32_tcgen05(C.c_int64(n), C.c_int(p), _ptr(X), C.c_int(X.stride(0)), C.c_int(q),
                                         _ptr(Y), C.c_int(Y.stride(0)), _ptr(Cm), _stream(stream)))
    return Cm.t()


def gram_df(X, Y, stream=None):
    """C = X^T Y of FP64 row-major CUDA blocks (one aligned row stride) in double-float
    arithmetic (the FP64 refinement's Gram)."""
    torch = _torch()
    n, p = X.shape
    q = Y.shape[1]
    Cm = torch.empty((q, p), dtype=torch.float64, device=X.device)
    _check(lib().lobpcg_gram_f64_df(C.c_int64(n), C.c_int(p), _ptr(X), C.c_int(X.stride(0)), C.c_int(q), _ptr(Y),
                                    C.c_int(Y.stride(0)), _ptr(Cm), _stream(stream)))
    return Cm.t()


def update_f64_df(V, U, q=None, alpha=1.0, AV=None, base=None, X=None, AX=None, lam=None, resnorm=False,
                  stream=None):
    """FP64 block update X = base + alpha [V_0 ..] U (and AX, residual norms) in double-float
    arithmetic; the FP64 counterpart of update_f32 (same arguments, float64 blocks)."""
    torch = _torch()
    V = list(V)
    n = V[0].shape[0]
    ws = [int(v.shape[1]) for v in V]
    ld = int(V[0].stride(0))
    q = int(U.shape[1]) if q is None else int(q)
    if X is None:
        X = torch.empty((n, q), dtype=torch.float64, device=V[0].device)
    if AV is not None and AX is None:
        AX = torch.empty_like(X)
    Ucol = U if (U.stride(0) == 1 and U.stride(1) == U.shape[0]) else U.t().contiguous().t()
    vp = (C.c_void_p * len(V))(*[v.data_ptr() for v in V])
    ap = (C.c_void_p * len(V))(*[a.data_ptr() for a in AV]) if AV is not None else None
    warr = (C.c_int * len(V))(*ws)
    rn = (C.c_double * q)() if resnorm else None
    _check(lib().lobpcg_update_f64_df(C.c_int64(n), C.c_int(len(V)), vp, ap, warr, C.c_int(ld), _ptr(Ucol),
                                      C.c_int(q), C.c_double(alpha), _ptr(base),
                                      C.c_int(base.stride(0) if base is not None else 0), _ptr(X), _ptr(AX),
                                      C.c_int(X.stride(0)), _ptr(lam), rn, _stream(stream)))
    if AV is None:
        return X
    if resnorm:
        return X, AX, np.array(rn[:])
    return X, AX


def gram_noalloc(X, Y, out=None, stream=None):
    """C = X^T Y through the entry point that allocates no device memory itself.

    ``out`` may be a preallocated (q, p) float64 CUDA tensor (column-major storage of the
    p x q result); its transpose is returned.
    """
    torch = _torch()
    n, p = X.shape
    q = Y.shape[1]
    Cm = torch.empty((q, p), dtype=torch.float64, device=X.device) if out is None else out
    _check(lib().lobpcg_gram_f64_noalloc(C.c_int64(n), C.c_int(p), _ptr(X), C.c_int(X.stride(0)), C.c_int(q),
                                         _ptr(Y), C.c_int(Y.stride(0)), _ptr(Cm), _stream(stream)))
    return Cm.t()


def syev(a, two_stage=False, tol=0.0, stream=None):
    """Eigenvalues (ascending) and eigenvectors of symmetric a; two_stage selects the
    FP32-then-FP64 Jacobi used by the FP32 phase of the mixed form, stopped at tol (0: 1e-15)."""
    torch = _torch()
    s = a.shape[0]
    ac = a.t().contiguous()  # column-major storage of a
    lam = torch.empty(s, dtype=torch.float64, device=a.device)
    U = torch.empty((s, s), dtype=torch.float64, device=a.device)
    if two_stage:
        _check(lib().lobpcg_syev2_f64(C.c_int(s), _ptr(ac), C.c_double(tol), _ptr(lam), _ptr(U), _stream(stream)))
    else:
        _check(lib().lobpcg_syev_f64(C.c_int(s), _ptr(ac), _ptr(lam), _ptr(U), _stream(stream)))
    return lam, U.t()


def ortho(X, tau=1e-14, cap=6, stream=None):
    """Algorithm 2 in place on a row-major block; returns (X, stats)."""
    n, p = X.shape
    st = (C.c_int * 4)()
    _check(lib().lobpcg_ortho_f64(C.c_int64(n), C.c_int(p), _ptr(X), C.c_int(X.stride(0)), C.c_double(tau),
                                  C.c_int(cap), st, _stream(stream)))
    return X, dict(passes=st[0], shifts=st[1], svqb=st[2], cap_hit=st[3])


def ortho_against(X, Y, tau=1e-14, cap=6, cap2=4, stream=None):
    """Algorithm 3 in place; returns (X, stats)."""
    n, p = X.shape
    q = 0 if Y is None else Y.shape[1]
    st = (C.c_int * 5)()
    _check(lib().lobpcg_ortho_against_f64(C.c_int64(n), C.c_int(p), _ptr(X), C.c_int(X.stride(0)), C.c_int(q),
                                          _ptr(Y), C.c_int(Y.stride(0) if q else 1), C.c_double(tau), C.c_int(cap),
                                          C.c_int(cap2), st, _stream(stream)))
    return X, dict(passes=st[0], cholqr_passes_max=st[1], shifts=st[2], svqb=st[3], cap_hits=st[4])


def upload_csr(a, device="cuda"):
    """Copy a synth.CSR-like matrix (numpy arrays) to CUDA tensors (no arithmetic)."""
    torch = _torch()
    return dict(row_ptr=torch.from_numpy(np.ascontiguousarray(a.row_ptr, dtype=np.int64)).to(device),
                col_idx=torch.from_numpy(np.ascontiguousarray(a.col_idx, dtype=np.int32)).to(device),
                val=torch.from_numpy(np.ascontiguousarray(a.val, dtype=np.float64)).to(device),
                diag=torch.from_numpy(np.ascontiguousarray(a.diag, dtype=np.float64)).to(device))


# ------------------------------------------------------------------ learned preconditioner

def mlp_num_params() -> int:
    return lib().lobpcg_mlp_num_params()


def mlp_forward(F, params, bf16=True, stream=None):
    """s = softplus(MLP(F)) for features F (N x 3 float32 CUDA) and float32 parameters."""
    torch = _torch()
    s = torch.empty(F.shape[0], dtype=torch.float32, device=F.device)
    _check(lib().lobpcg_mlp_forward(C.c_int64(F.shape[0]), _ptr(F), _ptr(params), _ptr(s), C.c_int(int(bf16)),
                                    _stream(stream)))
    return s


def mlp_backward(F, params, g, grad, bf16=True, stream=None):
    """grad += sum_i g_i ds_i/dparams (in place)."""
    _check(lib().lobpcg_mlp_backward(C.c_int64(F.shape[0]), _ptr(F), _ptr(params), _ptr(g), _ptr(grad),
                                     C.c_int(int(bf16)), _stream(stream)))
    return grad


def mlp_loss(col, q, e, s, far_we, far_ww, ee, stream=None):
    """Returns (mean column loss as a float, dL/ds CUDA tensor)."""
    torch = _torch()
    ncol = ee.numel()
    work = torch.empty(2 * ncol, dtype=torch.float64, device=q.device)
    loss = torch.empty(1, dtype=torch.float64, device=q.device)
    d = torch.empty_like(s)
    _check(lib().lobpcg_mlp_loss(C.c_int64(s.numel()), C.c_int(ncol), _ptr(col), _ptr(q), _ptr(e), _ptr(s),
                                 _ptr(far_we), _ptr(far_ww), _ptr(ee), _ptr(work), _ptr(d), _ptr(loss),
                                 _stream(stream)))
    return float(loss.item()), d


def mlp_adam(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().lobpcg_mlp_adam(C.c_int(params.numel()), _ptr(params), _ptr(grad), _ptr(m), _ptr(v), C.c_int(step),
                                 C.c_float(lr), C.c_float(beta1), C.c_float(beta2), C.c_float(eps), _stream(stream)))


def row_norms(diag_n, row_ptr=None, col_idx=None, val=None, dense=None, stream=None):
    """(rho, mean rho): off-diagonal 2-norms of the rows of A."""
    torch = _torch()
    n = diag_n
    rho = torch.empty(n, dtype=torch.float32, device="cuda")
    mean = C.c_double(0.0)
    At = None if dense is None else (dense if dense.t().is_contiguous() else dense.t().contiguous().t())
    _check(lib().lobpcg_row_norms(C.c_int64(n), _ptr(row_ptr), _ptr(col_idx), _ptr(val), _ptr(At), C.c_int64(n),
                                  _ptr(rho), C.byref(mean), _stream(stream)))
    return rho, mean.value


def precond_features(X, AX, lam, diag, rho, cscale, colmax, XS, alpha, stream=None):
    """Training features of a row-major block (see lobpcg_precond_features)."""
    torch = _torch()
    n, p = X.shape
    dev = X.device
    F = torch.empty((n * p, 3), dtype=torch.float32, device=dev)
    q = torch.empty(n * p, dtype=torch.float32, device=dev)
    e = torch.empty(n * p, dtype=torch.float32, device=dev)
    near = torch.empty(n * p, dtype=torch.int32, device=dev)
    sums = torch.empty(3 * p, dtype=torch.float64, device=dev)
    _check(lib().lobpcg_precond_features(C.c_int64(n), C.c_int(p), _ptr(X), _ptr(AX), C.c_int(X.stride(0)),
                                         _ptr(lam), _ptr(diag), _ptr(rho), C.c_float(cscale), _ptr(colmax), _ptr(XS),
                                         _ptr(alpha), _ptr(F), _ptr(q), _ptr(e), _ptr(near), _ptr(sums),
                                         _stream(stream)))
    return F, q, e, near, sums[:p], sums[p:2 * p], sums[2 * p:]


def load_mlp_weights(path=None):
    """The trained parameters shipped with the package (float32 numpy array)."""
    p = pathlib.Path(path) if path else _HERE / "weights" / "precond_mlp.npy"
    return np.load(p).astype(np.float32)


def solve_batched(solvers, ks, tols, X0s=None, nthreads=32):
    """Solve independent problems concurrently (lobpcg_solve_batched).

    solvers: list of Solver (each with its own CUDA stream); ks, tols: per problem;
    X0s: optional list of initial blocks (CUDA float64, n x (k + extra)) or None.
    Returns a list of Result in problem order."""
    torch = _torch()
    nprob = len(solvers)
    ctxs = (C.c_void_p * nprob)(*[s.handle.value for s in solvers])
    karr = (C.c_int * nprob)(*ks)
    tarr = (C.c_double * nprob)(*tols)
    keep = []
    x0p = None
    if X0s is not None:
        cols = []
        for s, k, X in zip(solvers, ks, X0s):
            if X is None:
                cols.append(None)
                continue
            Xc = X.t().contiguous().t()
            keep.append(Xc)
            cols.append(Xc.data_ptr())
        x0p = (C.c_void_p * nprob)(*cols)
    evals = [np.zeros(k) for k in ks]
    res = [np.zeros(k) for k in ks]
    vecs = [torch.empty((k, s.n), dtype=torch.float64, device="cuda").t() for s, k in zip(solvers, ks)]
    ev_p = (C.c_void_p * nprob)(*[e.ctypes.data for e in evals])
    rs_p = (C.c_void_p * nprob)(*[r.ctypes.data for r in res])
    vc_p = (C.c_void_p * nprob)(*[v.data_ptr() for v in vecs])
    infos = (_Info * nprob)()
    st = (C.c_int * nprob)()
    torch.cuda.synchronize()
    lib().lobpcg_solve_batched(ctxs, C.c_int(nprob), karr, tarr, x0p, ev_p, vc_p, rs_p, infos, st, C.c_int(nthreads))
    out = []
    for i in range(nprob):
        d = {f: getattr(infos[i], f) for f, _ in _Info._fields_}
        d["phase_seconds"] = dict(zip(PHASES, list(infos[i].phase_seconds)))
        d["phase_seconds_fp64"] = dict(zip(PHASES, list(infos[i].phase_seconds_fp64)))
        if st[i] not in (OK, ENOCONV):
            raise LobpcgError(st[i], lib().lobpcg_last_error(solvers[i].handle).decode())
        out.append(Result(st[i], evals[i], vecs[i], res[i], d))
    return out
