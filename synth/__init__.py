"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws random numbers and assembles matrices; it holds none of the
eigensolver's arithmetic.  Every generator takes an explicit seed and uses numpy's
counter-based Philox4x32-10 bit generator, so a (recipe, seed) pair always yields the
same bytes on any machine.

The recipes stand in for the paper's quantum-chemistry matrices (Sec. 4: Full-CI
Hamiltonians, SCF/CASSCF orbital Hessians), which are not available:

* ``sparse_cfg1``: diagonally dominant sparse matrix, diagonal 0.01*i + U(0, 0.005)
  sorted ascending, 16 random off-diagonal positions per row mirrored, values N(0, 0.01^2).
* ``sparse_ci``: CI-like banded matrix, diagonal 0.001*i + U(0, 0.01), per row 28
  distinct couplings inside (i, i+256] plus 4 long-range couplings in (i, n), mirrored,
  values N(0, 0.005^2)  (about 64 off-diagonals per row).
* ``dense_casscf``: dense ill-conditioned matrix D + U S U^T, D log-uniform in
  [1e-3, 1e2], U an orthonormalised n x r Gaussian, S uniform in [-5, 5].
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Philox4x32-10 generator keyed by (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream)]))


@dataclasses.dataclass
class CSR:
    """Symmetric matrix in CSR form: int64 row_ptr (n+1), int32 col_idx, float64 val."""

    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray
    diag: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.n, self.n))


def _assemble(n: int, diag: np.ndarray, i: np.ndarray, j: np.ndarray, v: np.ndarray) -> CSR:
    """Mirror the strict upper-triangle triplets (i < j), add the diagonal, sort each row."""
    rows = np.concatenate([i, j, np.arange(n, dtype=np.int64)])
    cols = np.concatenate([j, i, np.arange(n, dtype=np.int64)])
    vals = np.concatenate([v, v, diag])
    m = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    m.sum_duplicates()
    m.sort_indices()
    return CSR(n=n, row_ptr=m.indptr.astype(np.int64), col_idx=m.indices.astype(np.int32),
               val=m.data.astype(np.float64), diag=diag.astype(np.float64))


def _dedupe_first(i: np.ndarray, j: np.ndarray, v: np.ndarray, n: int):
    """Keep the first occurrence (in generation order) of every unordered pair."""
    lo = np.minimum(i, j)
    hi = np.maximum(i, j)
    key = lo * np.int64(n) + hi
    _, first = np.unique(key, return_index=True)
    first.sort()
    return lo[first], hi[first], v[first]


def sparse_cfg1(n: int = 4096, seed: int = 0, per_row: int = 16, sigma: float = 0.01,
                step: float = 0.01, jitter: float = 0.005) -> CSR:
    """Diagonally dominant sparse matrix (the n=4096, k=4 parity workload's recipe)."""
    g = rng(seed, 1)
    diag = np.sort(step * np.arange(n) + g.uniform(0.0, jitter, size=n))
    i = np.repeat(np.arange(n, dtype=np.int64), per_row)
    # j uniform over the n-1 indices other than i
    r = g.integers(0, n - 1, size=n * per_row, dtype=np.int64)
    j = np.where(r >= i, r + 1, r)
    v = g.normal(0.0, sigma, size=n * per_row)
    lo, hi, vv = _dedupe_first(i, j, v, n)
    return _assemble(n, diag, lo, hi, vv)


def sparse_ci(n: int = 2_000_000, seed: int = 0, band: int = 256, per_band: int = 28,
              long_range: int = 4, sigma: float = 0.005, chunk: int = 1 << 16) -> CSR:
    """CI-like banded sparse matrix (the n=2,000,000, k=16 workload's recipe)."""
    g = rng(seed, 2)
    diag = 0.001 * np.arange(n) + g.uniform(0.0, 0.01, size=n)
    ii, jj = [], []
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        rows = np.arange(r0, r1, dtype=np.int64)
        width = np.minimum(band, n - 1 - rows)  # admissible offsets 1..width
        keys = g.random((r1 - r0, band), dtype=np.float32)
        keys[np.arange(band)[None, :] >= width[:, None]] = np.inf
        take = min(per_band, band)
        pos = np.argpartition(keys, take - 1, axis=1)[:, :take]
        ok = pos < width[:, None]
        off = pos + 1
        ii.append(np.broadcast_to(rows[:, None], off.shape)[ok])
        jj.append((rows[:, None] + off)[ok])
        # long-range partners uniform in (i, n)
        span = (n - 1 - rows).astype(np.float64)
        u = g.random((r1 - r0, long_range))
        lr = rows[:, None] + 1 + np.floor(u * span[:, None]).astype(np.int64)
        okl = span[:, None] > 0
        okl = np.broadcast_to(okl, lr.shape)
        ii.append(np.broadcast_to(rows[:, None], lr.shape)[okl])
        jj.append(lr[okl])
    i = np.concatenate(ii)
    j = np.concatenate(jj)
    # chunk order keeps band entries of a row before its long-range entries
    order = np.argsort(i, kind="stable")
    i, j = i[order], j[order]
    v = g.normal(0.0, sigma, size=i.size)
    lo, hi, vv = _dedupe_first(i, j, v, n)
    return _assemble(n, diag, lo, hi, vv)


def dense_casscf(n: int = 8192, seed: int = 0, rank: int = 256) -> tuple[np.ndarray, np.ndarray]:
    """Dense symmetric D + U S U^T (column-major == row-major since exactly symmetric)."""
    g = rng(seed, 3)
    d = 10.0 ** g.uniform(-3.0, 2.0, size=n)
    q, _ = np.linalg.qr(g.standard_normal((n, rank)))
    s = g.uniform(-5.0, 5.0, size=rank)
    a = (q * s) @ q.T
    a = 0.5 * (a + a.T)
    a[np.diag_indices(n)] += d
    return np.asfortranarray(a), np.ascontiguousarray(np.diag(a)).copy()


def diag_guess(diag: np.ndarray, m: int, seed: int, noise: float = 1e-3) -> np.ndarray:
    """Initial block: unit vectors at the m smallest diagonal entries plus N(0, noise^2).

    Returned as an n x m column-major (Fortran-ordered) float64 array.  noise=0 gives the
    plain unit-vector guess used for the large CI-like matrices, where per-entry noise
    over millions of rows would dominate the Rayleigh quotient.
    """
    n = diag.shape[0]
    g = rng(seed, 4)
    if noise > 0:
        x = g.normal(0.0, noise, size=(m, n)).T.copy(order="F")
    else:
        x = np.zeros((n, m), order="F")
    idx = np.argsort(diag, kind="stable")[:m]
    x[idx, np.arange(m)] += 1.0
    return x


def gaussian_block(n: int, m: int, seed: int) -> np.ndarray:
    """n x m column-major block of independent N(0, 1) entries."""
    g = rng(seed, 5)
    return g.standard_normal((m, n)).T.copy(order="F")


def tridiag_toeplitz(n: int, a: float, b: float) -> CSR:
    """Tridiagonal Toeplitz matrix with diagonal a and off-diagonals b."""
    i = np.arange(n - 1, dtype=np.int64)
    return _assemble(n, np.full(n, float(a)), i, i + 1, np.full(n - 1, float(b)))


def random_sparse_sym(n: int, per_row: int, seed: int, diag_scale: float = 1.0,
                      sigma: float = 1.0) -> CSR:
    """Generic random sparse symmetric matrix (not diagonally dominant unless asked)."""
    g = rng(seed, 6)
    diag = diag_scale * g.standard_normal(n)
    i = np.repeat(np.arange(n, dtype=np.int64), per_row)
    r = g.integers(0, n - 1, size=n * per_row, dtype=np.int64)
    j = np.where(r >= i, r + 1, r)
    v = g.normal(0.0, sigma, size=n * per_row)
    lo, hi, vv = _dedupe_first(i, j, v, n)
    return _assemble(n, diag, lo, hi, vv)


def dense_from_csr(a: CSR) -> np.ndarray:
    return np.asfortranarray(a.to_scipy().toarray())


def sparse_cfg1_torch(n: int, seed: int, device="cuda", per_row: int = 16, sigma: float = 0.01,
                      step: float = 0.01, jitter: float = 0.005):
    """The cfg1 recipe generated on the GPU with torch's seeded Philox generator.

    Same construction as sparse_cfg1 (diagonal step*i + U(0, jitter) sorted, per_row random
    couplings j != i per row, unordered pairs deduplicated keeping the first, mirrored,
    N(0, sigma^2)), for the large batched workload where host generation would take
    minutes.  Returns CUDA tensors (row_ptr int64, col_idx int32, val float64, diag float64).
    The random stream differs from the numpy one, so the matrices differ from sparse_cfg1.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    ar = torch.arange(n, device=device, dtype=torch.int64)
    diag = torch.sort(step * ar.double() + jitter * torch.rand(n, generator=g, device=device, dtype=torch.float64)).values
    i = ar.repeat_interleave(per_row)
    r = torch.randint(0, n - 1, (n * per_row,), generator=g, device=device, dtype=torch.int64)
    j = torch.where(r >= i, r + 1, r)
    v = sigma * torch.randn(n * per_row, generator=g, device=device, dtype=torch.float64)
    lo, hi = torch.minimum(i, j), torch.maximum(i, j)
    key = lo * n + hi
    # first occurrence of every key in generation order
    sk, perm = torch.sort(key, stable=True)
    first = torch.ones_like(sk, dtype=torch.bool)
    first[1:] = sk[1:] != sk[:-1]
    keep = perm[first]
    keep, _ = torch.sort(keep)
    lo, hi, v = lo[keep], hi[keep], v[keep]
    rows = torch.cat([lo, hi, ar])
    cols = torch.cat([hi, lo, ar])
    vals = torch.cat([v, v, diag])
    order = torch.argsort(rows * n + cols)
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = torch.bincount(rows, minlength=n)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return dict(row_ptr=row_ptr, col_idx=cols.to(torch.int32).contiguous(), val=vals.contiguous(), diag=diag)


def batched_specs(nprob: int = 256, seed: int = 0, n_range=(10_000, 500_000), k_range=(1, 32)):
    """(n, k, seed) of the batched serving workload: n ~ U[n_range], k ~ U{k_range}."""
    g = rng(seed, 7)
    ns = g.integers(n_range[0], n_range[1] + 1, size=nprob)
    ks = g.integers(k_range[0], k_range[1] + 1, size=nprob)
    return [(int(n), int(k), int(seed) * 100_000 + p) for p, (n, k) in enumerate(zip(ns, ks))]


def diag_guess_torch(diag, m: int):
    """Unit vectors at the m smallest diagonal entries (n x m float64 on diag's device)."""
    import torch
    n = diag.numel()
    idx = torch.argsort(diag, stable=True)[:m]
    x = torch.zeros((n, m), dtype=torch.float64, device=diag.device)
    x[idx, torch.arange(m, device=diag.device)] = 1.0
    return x
