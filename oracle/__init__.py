"""CPU FP64 oracle of the LOBPCG method (arXiv 2305.06668, Algorithms 1-3).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, by ``__graft_entry__.smoke()`` and by
the CPU-baseline leg of ``bench.py``; never by the GPU package.  The C source it wraps
is plain, slow FP64 code that follows the paper's algorithms step by step.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np

from . import build as _build

_lib = None


class _Matrix(C.Structure):
    _fields_ = [("n", C.c_int64), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("val", C.c_void_p), ("dense", C.c_void_p), ("ld", C.c_int64)]


class _Opts(C.Structure):
    _fields_ = [("k", C.c_int), ("extra", C.c_int), ("maxiter", C.c_int), ("tol_kind", C.c_int),
                ("precond", C.c_int), ("ortho_cap", C.c_int), ("ortho2_cap", C.c_int),
                ("tol", C.c_double), ("tau", C.c_double), ("trim", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("cholqr_passes_max", C.c_int),
                ("ortho_passes_max", C.c_int), ("shifts", C.c_int), ("svqb", C.c_int),
                ("cap_hits", C.c_int), ("spmm_columns", C.c_int), ("w_dropped", C.c_int),
                ("p_dropped", C.c_int), ("ortho_grams", C.c_int), ("skipped_recheck", C.c_int),
                ("skipped_test", C.c_int)]


class _OrthoStats(C.Structure):
    _fields_ = [("passes", C.c_int), ("grams", C.c_int), ("shifts", C.c_int), ("svqb", C.c_int),
                ("cap_hits", C.c_int), ("cholqr_passes_max", C.c_int), ("skipped_recheck", C.c_int),
                ("skipped_test", C.c_int)]


class _Hist(C.Structure):
    _fields_ = [("cap", C.c_int), ("lambda_", C.c_void_p), ("resnorm", C.c_void_p),
                ("m_act", C.c_void_p), ("rows", C.c_int), ("w_cols", C.c_void_p), ("p_cols", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(str(path))
        _lib.oracle_lobpcg.restype = C.c_int
        _lib.oracle_jacobi_eig.restype = C.c_int
        _lib.oracle_cholesky.restype = C.c_int
        _lib.oracle_ortho.restype = C.c_int
        _lib.oracle_ortho_against.restype = C.c_int
        _lib.oracle_threads.restype = C.c_int
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _f64(a) -> np.ndarray:
    return np.require(a, dtype=np.float64, requirements=["F", "A", "W"]).copy(order="F")


class Operator:
    """Keeps the arrays alive and exposes the C struct."""

    def __init__(self, csr=None, dense: np.ndarray | None = None):
        if dense is not None:
            self.dense = np.asfortranarray(dense, dtype=np.float64)
            self.n = self.dense.shape[0]
            self.s = _Matrix(self.n, None, None, None, _p(self.dense), self.n)
        else:
            self.row_ptr = np.ascontiguousarray(csr.row_ptr, dtype=np.int64)
            self.col_idx = np.ascontiguousarray(csr.col_idx, dtype=np.int32)
            self.val = np.ascontiguousarray(csr.val, dtype=np.float64)
            self.n = csr.n
            self.s = _Matrix(self.n, _p(self.row_ptr), _p(self.col_idx), _p(self.val), None, 0)


def _operator(A) -> Operator:
    if isinstance(A, Operator):
        return A
    if isinstance(A, np.ndarray):
        return Operator(dense=A)
    return Operator(csr=A)


def apply(A, X: np.ndarray) -> np.ndarray:
    op = _operator(A)
    X = _f64(X.reshape(op.n, -1))
    Y = np.zeros_like(X, order="F")
    lib().oracle_apply(C.byref(op.s), C.c_int(X.shape[1]), _p(X), _p(Y))
    return Y


def jacobi_eig(a: np.ndarray):
    a = _f64(a)
    s = a.shape[0]
    lam = np.zeros(s)
    U = np.zeros((s, s), order="F")
    sweeps = lib().oracle_jacobi_eig(C.c_int(s), _p(a), _p(lam), _p(U))
    return lam, U, sweeps


def cholesky(M: np.ndarray):
    L = _f64(M)
    fail = lib().oracle_cholesky(C.c_int(L.shape[0]), _p(L))
    return np.tril(L), fail


def gram(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    X = _f64(X)
    Y = _f64(Y)
    Cm = np.zeros((X.shape[1], Y.shape[1]), order="F")
    lib().oracle_gram(C.c_int64(X.shape[0]), C.c_int(X.shape[1]), _p(X), C.c_int(Y.shape[1]), _p(Y), _p(Cm))
    return Cm


def svqb(X: np.ndarray) -> np.ndarray:
    """One SVQB step (the fallback of Algorithm 2 when shifted Cholesky fails)."""
    X = _f64(X)
    M = gram(X, X)
    lib().oracle_svqb(C.c_int64(X.shape[0]), C.c_int(X.shape[1]), _p(X), _p(M))
    return X


def ortho(X: np.ndarray, tau: float = 1e-14, cap: int = 6, trim: bool = True):
    """Algorithm 2 (with trim: the re-check skip of reading R17).  Returns (Q, stats)."""
    X = _f64(X)
    st = _OrthoStats()
    passes = lib().oracle_ortho_ex(C.c_int64(X.shape[0]), C.c_int(X.shape[1]), _p(X), C.c_double(tau),
                                   C.c_int(cap), C.c_int(1 if trim else 0), C.byref(st))
    d = {f: getattr(st, f) for f, _ in _OrthoStats._fields_}
    d["passes"] = passes
    return X, d


def ortho_against(X: np.ndarray, Y: np.ndarray, tau: float = 1e-14, cap: int = 6, cap2: int = 4,
                  trim: bool = True):
    """Algorithm 3 (with trim: readings R17 and R18).  Returns (Q, stats)."""
    X = _f64(X)
    Y = _f64(Y)
    st = _OrthoStats()
    passes = lib().oracle_ortho_against_ex(C.c_int64(X.shape[0]), C.c_int(X.shape[1]), _p(X),
                                           C.c_int(Y.shape[1]), _p(Y), C.c_double(tau), C.c_int(cap),
                                           C.c_int(cap2), C.c_int(1 if trim else 0), C.byref(st))
    d = {f: getattr(st, f) for f, _ in _OrthoStats._fields_}
    d["passes"] = passes
    return X, d


@dataclasses.dataclass
class Result:
    status: int
    evals: np.ndarray
    evecs: np.ndarray
    resnorms: np.ndarray
    info: dict
    hist_lambda: np.ndarray
    hist_res: np.ndarray
    hist_mact: np.ndarray
    hist_wcols: np.ndarray
    hist_pcols: np.ndarray


def lobpcg(A, diag, k: int, X0: np.ndarray, tol: float = 1e-8, extra: int = 0, maxiter: int = 1000,
           tol_kind: int = 0, precond: int = 1, tau: float = 1e-14, ortho_cap: int = 6,
           ortho2_cap: int = 4, hist_cap: int | None = None, trim: bool = True) -> Result:
    """Algorithm 1 on a CSR (synth.CSR) or dense (ndarray) symmetric matrix.  trim: the cost
    trims of Sec. 3.2 (readings R17, R18), as in the GPU library's default; False runs the
    printed Algorithms 2 and 3."""
    op = _operator(A)
    n = op.n
    m = k + extra
    X0 = _f64(X0)
    assert X0.shape == (n, m), (X0.shape, n, m)
    d = None if diag is None else np.ascontiguousarray(diag, dtype=np.float64)
    opts = _Opts(k, extra, maxiter, tol_kind, precond, ortho_cap, ortho2_cap, tol, tau, 1 if trim else 0)
    evals = np.zeros(k)
    evecs = np.zeros((n, k), order="F")
    res = np.zeros(k)
    info = _Info()
    cap = (maxiter + 1) if hist_cap is None else hist_cap
    hl = np.zeros((cap, m))
    hr = np.zeros((cap, m))
    hm = np.zeros(cap, dtype=np.int32)
    hw = np.zeros(cap, dtype=np.int32)
    hp = np.zeros(cap, dtype=np.int32)
    hist = _Hist(cap, _p(hl), _p(hr), _p(hm), 0, _p(hw), _p(hp))
    st = lib().oracle_lobpcg(C.byref(op.s), _p(d), C.byref(opts), _p(X0), _p(evals), _p(evecs),
                             _p(res), C.byref(info), C.byref(hist))
    info_d = {f: getattr(info, f) for f, _ in _Info._fields_}
    r = hist.rows
    return Result(st, evals, evecs, res, info_d, hl[:r], hr[:r], hm[:r], hw[:r], hp[:r])


def precondition(R: np.ndarray, lam: np.ndarray, diag: np.ndarray, m_conv: int, m_act: int,
                 precond: int = 1) -> np.ndarray:
    """W~ = T R over the active columns m_conv .. m_conv + m_act - 1 (reading R6)."""
    R = _f64(R)
    n = R.shape[0]
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    diag = np.ascontiguousarray(diag, dtype=np.float64)
    W = np.zeros((n, max(m_act, 1)), order="F")
    lib().oracle_precondition(C.c_int64(n), C.c_int(m_conv), C.c_int(m_act), _p(R), _p(lam), _p(diag),
                              C.c_int(precond), _p(W))
    return W[:, :m_act]


def tridiag_solve(dl: np.ndarray, d: np.ndarray, du: np.ndarray, shift: float, b: np.ndarray) -> np.ndarray:
    """x = (T - shift I)^{-1} b for the tridiagonal T = (dl, d, du) (reading R24)."""
    d = _f64(d)
    n = d.shape[0]
    dl = _f64(dl) if n > 1 else np.zeros(1)
    du = _f64(du) if n > 1 else np.zeros(1)
    b = _f64(b)
    x = np.zeros(n)
    lib().oracle_tridiag_solve(C.c_int64(n), _p(dl), _p(d), _p(du), C.c_double(shift), _p(b), _p(x))
    return x


def tridiag_of(A) -> tuple[np.ndarray, np.ndarray]:
    """(dl, du): the first sub- and super-diagonals of A (CSR or dense)."""
    op = _operator(A)
    n = op.n
    dl = np.zeros(max(n - 1, 1))
    du = np.zeros(max(n - 1, 1))
    lib().oracle_tridiag_of(C.byref(op.s), _p(dl), _p(du))
    return dl[: max(n - 1, 0)], du[: max(n - 1, 0)]


def precondition_tridiag(R: np.ndarray, lam: np.ndarray, dl: np.ndarray, diag: np.ndarray, du: np.ndarray,
                         m_conv: int, m_act: int) -> np.ndarray:
    """W[:, c] = (T - lam[m_conv + c] I)^{-1} R[:, m_conv + c] (reading R24)."""
    R = np.asfortranarray(_f64(R))
    n = R.shape[0]
    W = np.zeros((n, m_act), order="F")
    dl = _f64(dl) if n > 1 else np.zeros(1)
    du = _f64(du) if n > 1 else np.zeros(1)
    lib().oracle_precondition_tridiag(C.c_int64(n), C.c_int(m_conv), C.c_int(m_act), _p(R), _p(_f64(lam)),
                                      _p(dl), _p(_f64(diag)), _p(du), _p(W))
    return W


def drop_unorthogonal_columns(W: np.ndarray, Y: np.ndarray | None, tau: float = 1e-14,
                              check_norm: bool = True) -> np.ndarray:
    """Reading R16: the columns of W kept (packed, in order)."""
    W = _f64(W)
    n, p = W.shape
    q = 0 if Y is None else Y.shape[1]
    Yf = None if Y is None else _f64(Y)
    lib().oracle_drop_unorthogonal_columns.restype = C.c_int
    kept = lib().oracle_drop_unorthogonal_columns(C.c_int64(n), C.c_int(p), _p(W), C.c_int(q), _p(Yf),
                                                  C.c_double(tau), C.c_int(1 if check_norm else 0))
    return W[:, :kept]


def lobpcg_gen(A, B, dA, dB, k: int, X0: np.ndarray, tol: float = 1e-8, extra: int = 0, maxiter: int = 1000,
               tol_kind: int = 0, precond: int = 1, tau: float = 1e-14, ortho_cap: int = 6,
               ortho2_cap: int = 4, hist_cap: int | None = None, trim: bool = True) -> Result:
    """Algorithm 1 for A x = lambda B x (Sec. 3.3); A, B CSR (synth.CSR) or dense ndarrays."""
    opA, opB = _operator(A), _operator(B)
    n = opA.n
    m = k + extra
    X0 = _f64(X0)
    assert X0.shape == (n, m), (X0.shape, n, m)
    da = None if dA is None else np.ascontiguousarray(dA, dtype=np.float64)
    db = None if dB is None else np.ascontiguousarray(dB, dtype=np.float64)
    opts = _Opts(k, extra, maxiter, tol_kind, precond, ortho_cap, ortho2_cap, tol, tau, 1 if trim else 0)
    evals = np.zeros(k)
    evecs = np.zeros((n, k), order="F")
    res = np.zeros(k)
    info = _Info()
    cap = (maxiter + 1) if hist_cap is None else hist_cap
    hl, hr = np.zeros((cap, m)), np.zeros((cap, m))
    hm, hw, hp = (np.zeros(cap, dtype=np.int32) for _ in range(3))
    hist = _Hist(cap, _p(hl), _p(hr), _p(hm), 0, _p(hw), _p(hp))
    lib().oracle_lobpcg_gen.restype = C.c_int
    st = lib().oracle_lobpcg_gen(C.byref(opA.s), C.byref(opB.s), _p(da), _p(db), C.byref(opts), _p(X0),
                                 _p(evals), _p(evecs), _p(res), C.byref(info), C.byref(hist))
    info_d = {f: getattr(info, f) for f, _ in _Info._fields_}
    r = hist.rows
    return Result(st, evals, evecs, res, info_d, hl[:r], hr[:r], hm[:r], hw[:r], hp[:r])


def threads() -> int:
    return lib().oracle_threads()


# ------------------------------------------------------------------ learned preconditioner scale

def mlp_num_params() -> int:
    lib().oracle_mlp_num_params.restype = C.c_int
    return lib().oracle_mlp_num_params()


def mlp_forward(P: np.ndarray, F: np.ndarray) -> np.ndarray:
    """s = softplus(MLP(f)) for features F (N x 3) and parameters P (float64)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    s = np.zeros(F.shape[0])
    lib().oracle_mlp_forward(_p(P), C.c_int64(F.shape[0]), _p(F), _p(s))
    return s


def mlp_backward(P: np.ndarray, F: np.ndarray, g: np.ndarray) -> np.ndarray:
    """sum_i g_i ds_i/dP."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    grad = np.zeros_like(P)
    lib().oracle_mlp_backward(_p(P), C.c_int64(F.shape[0]), _p(F), _p(g), _p(grad))
    return grad


def mlp_loss(col, q, e, s, far_we, far_ww, ee):
    """Mean over columns of 1 - cos^2(w, e) with w = s q; returns (loss, dL/ds)."""
    col = np.ascontiguousarray(col, dtype=np.int32)
    q, e, s = (np.ascontiguousarray(v, dtype=np.float64) for v in (q, e, s))
    far_we, far_ww, ee = (np.ascontiguousarray(v, dtype=np.float64) for v in (far_we, far_ww, ee))
    d = np.zeros_like(s)
    lib().oracle_mlp_loss.restype = C.c_double
    loss = lib().oracle_mlp_loss(C.c_int64(len(s)), C.c_int(len(ee)), _p(col), _p(q), _p(e), _p(s), _p(far_we),
                                 _p(far_ww), _p(ee), _p(d))
    return loss, d
