"""The tridiagonal preconditioner (Sec. 4.4, reading R24) on the GPU against the oracle.

The GPU solve is partitioned (blocks of 32 to 1024 rows, coupled through their end
unknowns) and runs in FP32, so it is compared with the oracle's FP64 solve through the FP32 error bounds:
a normwise backward error (residual) of 1e-5 and a forward error of 1e-5 times a bound on
the condition number of T - shift I.  Inside LOBPCG a preconditioner only shapes the
search direction: the solver's eigenvalues must meet |d lambda| <= 1e-10 max(1, |lambda|),
and its eigenvectors, reached by another path than the oracle's, the Davis-Kahan bound."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import cuda, dev
from tests.util import cluster_angles, rel_eig_err

pytestmark = pytest.mark.gpu


def _gpu(torch, dl, d, du, shift, R):
    import paper_2305_06668_gb300 as lb
    n = d.size
    args = [dev(torch, dl if n > 1 else np.zeros(1)), dev(torch, d), dev(torch, du if n > 1 else np.zeros(1))]
    return lb.precond_tridiag(*args, dev(torch, shift), dev(torch, R)).cpu().numpy()


def _dense(dl, d, du, s):
    return np.diag(d - s) + np.diag(dl, -1) + np.diag(du, 1)


def _matvec(dl, d, du, s, x):
    y = (d - s) * x
    y[1:] += dl * x[:-1]
    y[:-1] += du * x[1:]
    return y


@pytest.mark.parametrize("n,p", [(1, 1), (2, 3), (1023, 7), (1024, 21), (1025, 5), (4097, 21), (100_003, 8)])
def test_diagonally_dominant_systems(n, p):
    """|d - shift| >= 2.5 > |dl| + |du|: kappa_inf <= (4.5 + 2) / (2.5 - 2) = 13.  Sizes span
    one partition, ragged tails (down to a one-row last partition at n = 1025) and
    thousands of partitions."""
    torch = cuda()
    g = np.random.default_rng(n + p)
    d = 3.0 + g.random(n)
    dl, du = g.uniform(-1, 1, max(n - 1, 0)), g.uniform(-1, 1, max(n - 1, 0))
    shift = g.uniform(-0.5, 0.5, p)
    R = g.normal(0, 1, (n, p))
    W = _gpu(torch, dl, d, du, shift, R)
    for j in range(p):
        ref = oracle.tridiag_solve(dl, d, du, shift[j], R[:, j])
        assert np.max(np.abs(W[:, j] - ref)) <= 1e-5 * 13 * np.max(np.abs(ref))
        res = _matvec(dl, d, du, shift[j], W[:, j]) - R[:, j]
        assert np.max(np.abs(res)) <= 1e-5 * (6.5 * np.max(np.abs(W[:, j])) + np.max(np.abs(R[:, j])))


def test_indefinite_systems_with_row_interchanges():
    """Diagonal of random sign (|d| in [0.5, 1.5]), off-diagonals N(0, 0.6^2): the elimination
    interchanges rows wherever |d - shift| < |dl|.  n = 3000: 94 partitions of 32 rows, the
    last one ragged.  Forward error against the oracle within 1e-5 kappa(T - shift I)."""
    torch = cuda()
    g = np.random.default_rng(11)
    n, p = 3000, 5
    d = g.choice([-1.0, 1.0], n) * g.uniform(0.5, 1.5, n)
    dl, du = g.normal(0, 0.6, n - 1), g.normal(0, 0.6, n - 1)
    shift = 0.05 * np.arange(p)
    R = g.normal(0, 1, (n, p))
    W = _gpu(torch, dl, d, du, shift, R)
    swaps = 0
    for j in range(p):
        M = _dense(dl, d, du, shift[j])
        kappa = np.linalg.cond(M, np.inf)
        ref = oracle.tridiag_solve(dl, d, du, shift[j], R[:, j])
        assert np.max(np.abs(W[:, j] - ref)) <= 1e-5 * kappa * np.max(np.abs(ref))
        res = M @ W[:, j] - R[:, j]
        assert np.max(np.abs(res)) <= 1e-5 * kappa * (np.max(np.abs(M)) * np.max(np.abs(W[:, j])))
        swaps += np.count_nonzero(np.abs(d[:-1] - shift[j]) < np.abs(dl))
    assert swaps > 100  # the case does exercise the interchange branch


def test_zero_diagonal_needs_interchanges_everywhere():
    """T = tridiag(1, 0, 1), n = 4096 (even partitions, each nonsingular): without pivoting
    every first pivot is 0.  Integer data stay exact in FP32."""
    torch = cuda()
    n = 4096
    dl = du = np.ones(n - 1)
    d = np.zeros(n)
    x = np.arange(1.0, n + 1.0)
    b = _matvec(dl, d, du, 0.0, x)
    W = _gpu(torch, dl, d, du, np.zeros(1), b[:, None])
    assert np.max(np.abs(W[:, 0] - x)) <= 1e-6 * n


def test_zero_off_diagonals_give_the_diagonal_preconditioner():
    """dl = du = 0 reduces R24 to R6 (guard included): the GPU result equals the oracle's
    diagonal preconditioner to FP32 rounding (2 eps32 relative)."""
    torch = cuda()
    lam = np.array([0.25, 4.0])
    diag = np.array([0.25, 0.25 + 5e-9, 0.25 - 5e-9, 1.25, 4.0, 4.0 + 2e-8, 4.0 - 3e-8, 3.0] * 300)
    n = diag.size
    R = synth.gaussian_block(n, 2, seed=31)
    W = _gpu(torch, np.zeros(n - 1), diag, np.zeros(n - 1), lam, np.ascontiguousarray(R))
    ref = oracle.precondition(R, lam, diag, m_conv=0, m_act=2)
    assert np.max(np.abs(W - ref) / np.abs(ref)) <= 2 * np.finfo(np.float32).eps


def _solve(torch, a, k, x0, dense=None, **kw):
    import paper_2305_06668_gb300 as lb
    if dense is not None:
        s = lb.Solver(diag=dev(torch, np.diag(dense).copy()), dense=torch.from_numpy(np.asfortranarray(dense)).cuda(),
                      precond=lb.PREC_TRIDIAG, **kw)
    else:
        s = lb.Solver(**lb.upload_csr(a), precond=lb.PREC_TRIDIAG, **kw)
    r = s.solve(k, 1e-8, X0=torch.from_numpy(x0).cuda())
    s.close()
    return r


def _parity(res, ref, lam_more):
    """Eigenvalues to 1e-10; eigenvectors, reached by a different path (the FP32
    preconditioner), to the a-posteriori bound sin(angle) <= (||r|| + ||r_oracle||) / gap
    plus 1e-7 (Davis-Kahan), the gap taken from lam_more (eigenvalues beyond the block)."""
    assert np.max(rel_eig_err(res.evals, ref.evals)) <= 1e-10
    V = res.evecs.cpu().numpy()
    for j in range(len(ref.evals)):
        gap = min(abs(lam_more[j] - lam_more[i]) for i in range(len(lam_more)) if i != j)
        ang = float(cluster_angles(ref.evals[j:j + 1], ref.evecs[:, j:j + 1], V[:, j:j + 1])[0])
        assert ang <= 1e-7 + (res.resnorms[j] + ref.resnorms[j]) / gap, (j, ang, gap)


@pytest.mark.parametrize("mixed", [False, True])
def test_lobpcg_cfg1_matches_oracle(mixed):
    """cfg1 (n = 4096, k = 4, seed 0) with the tridiagonal preconditioner, FP64 and mixed."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    a = synth.sparse_cfg1(n=4096, seed=0)
    x0 = synth.diag_guess(a.diag, 4, seed=0)
    ref = oracle.lobpcg(a, a.diag, 4, x0, tol=1e-8, precond=3)
    more = oracle.lobpcg(a, a.diag, 6, synth.diag_guess(a.diag, 6, seed=0), tol=1e-9, maxiter=3000)
    res = _solve(torch, a, 4, x0, precision=lb.MIXED if mixed else lb.FP64)
    assert ref.status == 0 and res.status == 0 and more.status == 0
    _parity(res, ref, more.evals)
    assert np.max(res.resnorms) <= 1e-8


def test_lobpcg_perturbed_toeplitz_iterations_follow_the_oracle():
    """Where the tridiagonal part carries most of A (tridiag(-1, 2, -1) plus a sparse
    perturbation), the GPU solve with the FP32 tridiagonal preconditioner takes about the
    oracle's iteration count (123 here) and reaches its eigenpairs."""
    torch = cuda()
    import scipy.sparse as sp
    n, k = 400, 3
    g = np.random.default_rng(5)
    i = g.integers(0, n, 3 * n)
    j = np.clip(i + g.integers(2, 20, 3 * n), 0, n - 1)
    keep = np.abs(i - j) >= 2
    P = sp.coo_matrix((g.normal(0, 0.05, keep.sum()), (i[keep], j[keep])), shape=(n, n)).tocsr()
    M = (synth.tridiag_toeplitz(n, 2.0, -1.0).to_scipy() + P + P.T).tocsr()
    M.sort_indices()
    a = synth.CSR(n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64),
                  M.diagonal().astype(np.float64))
    x0 = synth.gaussian_block(n, k, seed=7)
    ref = oracle.lobpcg(a, a.diag, k, x0, tol=1e-8, maxiter=20000, precond=3)
    res = _solve(torch, a, k, x0, maxiter=20000)
    assert ref.status == 0 and res.status == 0
    _parity(res, ref, np.linalg.eigvalsh(M.toarray())[:k + 2])
    assert res.info["iterations"] <= 1.5 * ref.info["iterations"] + 5


def test_lobpcg_dense_mixed_matches_oracle():
    """Dense CASSCF-like recipe at n = 1024 (rank 64), k = 4, mixed precision."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    A, _ = synth.dense_casscf(n=1024, seed=3, rank=64)
    d = np.diag(A).copy()
    x0 = synth.diag_guess(d, 4, seed=3)
    ref = oracle.lobpcg(A, d, 4, x0, tol=1e-8, maxiter=5000, precond=3)
    res = _solve(torch, None, 4, x0, dense=A, precision=lb.MIXED, maxiter=5000)
    assert ref.status == 0 and res.status == 0
    _parity(res, ref, np.linalg.eigvalsh(A)[:6])
