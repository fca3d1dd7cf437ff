"""Pins of the oracle's tridiagonal preconditioner (Sec. 4.4, reading R24): the solve against
LAPACK's banded solver and a dense solve, a system that cannot be solved without row
interchanges, a closed form, the guard, and the reduction to the diagonal preconditioner
(R6) when the off-diagonals vanish; then LOBPCG with it."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import synth
from tests.util import rel_eig_err


def _dense(dl, d, du, shift):
    return np.diag(d - shift) + np.diag(dl, -1) + np.diag(du, 1)


def _banded(dl, d, du, shift):
    n = d.size
    ab = np.zeros((3, n))
    ab[0, 1:] = du
    ab[1] = d - shift
    ab[2, :-1] = dl
    return ab


@pytest.mark.parametrize("n", [1, 2, 3, 17, 500])
@pytest.mark.parametrize("shift", [0.0, 0.37, -2.5])
def test_solve_matches_lapack_and_dense(n, shift):
    """Random non-symmetric tridiagonal systems, indefinite after the shift: the solution
    equals LAPACK's banded solve with partial pivoting and a dense solve to rounding."""
    g = np.random.default_rng(100 + n)
    d, dl, du = g.normal(0, 1, n), g.normal(0, 1, max(n - 1, 0)), g.normal(0, 1, max(n - 1, 0))
    b = g.normal(0, 1, n)
    x = oracle.tridiag_solve(dl, d, du, shift, b)
    ref = sla.solve_banded((1, 1), _banded(dl, d, du, shift), b)
    T = _dense(dl, d, du, shift)
    cond = np.linalg.cond(T)
    assert np.max(np.abs(x - ref)) <= 1e-15 * cond * np.max(np.abs(ref)) + 1e-300
    assert np.max(np.abs(x - np.linalg.solve(T, b))) <= 1e-14 * cond * np.max(np.abs(ref))
    assert np.max(np.abs(T @ x - b)) <= 1e-14 * (np.max(np.abs(T)) * np.max(np.abs(x)) + np.max(np.abs(b)))


def test_solve_needs_row_interchanges():
    """Zero diagonal: without partial pivoting the first pivot is 0.  T = tridiag(1, 0, 1)
    of even order is nonsingular; T x = b must hold exactly (small integers)."""
    n = 10
    dl = np.ones(n - 1)
    du = np.ones(n - 1)
    d = np.zeros(n)
    x_true = np.arange(1.0, n + 1.0)
    b = _dense(dl, d, du, 0.0) @ x_true
    x = oracle.tridiag_solve(dl, d, du, 0.0, b)
    assert np.array_equal(x, x_true)


def test_solve_closed_form_toeplitz():
    """T = tridiag(-1, 2, -1) (the second difference) applied to x_i = i (i = 1..n) gives
    b = (0, ..., 0, n + 1): the solve returns x_i = i."""
    n = 40
    b = np.zeros(n)
    b[-1] = n + 1
    x = oracle.tridiag_solve(-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1), 0.0, b)
    assert np.max(np.abs(x - np.arange(1.0, n + 1.0))) <= 1e-12 * n


def test_zero_off_diagonals_equal_the_diagonal_preconditioner():
    """With dl = du = 0 the elimination has no work and every pivot is d_i - lambda with
    R6's guard, so R24 gives R6's result bit for bit, guard cases included."""
    lam = np.array([0.25, 4.0])
    diag = np.array([0.25, 0.25 + 5e-9, 0.25 - 5e-9, 1.25, 4.0, 4.0 + 2e-8, 4.0 - 3e-8, 3.0])
    n = diag.size
    R = synth.gaussian_block(n, 2, seed=31)
    z = np.zeros(n - 1)
    W3 = oracle.precondition_tridiag(R, lam, z, diag, z, m_conv=0, m_act=2)
    W1 = oracle.precondition(R, lam, diag, m_conv=0, m_act=2)
    assert np.array_equal(W3, W1)
    W3b = oracle.precondition_tridiag(R, lam, z, diag, z, m_conv=1, m_act=1)
    assert np.array_equal(W3b[:, 0], W1[:, 1])


def test_guard_on_a_singular_system():
    """T - shift I singular: d = (1, 1), off-diagonals 0 and shift 1 make both pivots 0; the
    guard replaces each by +1e-8 (shift 1: floor 1e-8 max(1, 1)), so x = b / 1e-8.  With a
    coupling the 2 x 2 [[0, 1], [1, 0]] needs an interchange and is solved exactly."""
    b = np.array([3.0, -2.0])
    x = oracle.tridiag_solve(np.zeros(1), np.ones(2), np.zeros(1), 1.0, b)
    assert np.array_equal(x, b / 1e-8)
    x2 = oracle.tridiag_solve(np.ones(1), np.ones(2), np.ones(1), 1.0, b)
    assert np.array_equal(x2, np.array([-2.0, 3.0]))


def test_tridiag_of_reads_the_first_off_diagonals():
    """dl, du of a CSR matrix and of its dense copy equal numpy's diagonals of the dense
    matrix (cfg1 recipe: only some rows have an entry next to the diagonal)."""
    a = synth.sparse_cfg1(n=300, seed=1)
    A = synth.dense_from_csr(a)
    for src in (a, A):
        dl, du = oracle.tridiag_of(src)
        assert np.array_equal(dl, np.diag(A, -1)) and np.array_equal(du, np.diag(A, 1))
    assert 0 < np.count_nonzero(np.diag(A, 1)) < 299


def test_precondition_tridiag_columns_use_their_own_ritz_value():
    """Column c of W solves with lambda_{m_conv + c} (each against tridiag_solve)."""
    a = synth.tridiag_toeplitz(50, 2.0, -0.7)
    dl, du = oracle.tridiag_of(a)
    R = synth.gaussian_block(50, 3, seed=4)
    lam = np.array([0.1, 0.5, 1.3])
    W = oracle.precondition_tridiag(R, lam, dl, a.diag, du, m_conv=1, m_act=2)
    for c in range(2):
        assert np.array_equal(W[:, c], oracle.tridiag_solve(dl, a.diag, du, lam[1 + c], R[:, 1 + c]))


def test_lobpcg_tridiagonal_beats_diagonal_on_a_perturbed_toeplitz():
    """A = tridiag(-1, 2, -1) + a sparse symmetric perturbation N(0, 0.05^2) at distances
    2..19 from the diagonal.  T - theta I is close to A - theta I, while the diagonal
    preconditioner is nearly a constant scale: the tridiagonal one needs at most 3/4 of
    the iterations (123 against 179 here), and both reach LAPACK's eigenvalues.  (With T = A exactly, the
    preconditioned residual (A - theta I)^{-1} r is x itself, already in the basis.)"""
    import scipy.sparse as sp
    n, k = 400, 3
    g = np.random.default_rng(5)
    i = g.integers(0, n, 3 * n)
    j = np.clip(i + g.integers(2, 20, 3 * n), 0, n - 1)
    keep = np.abs(i - j) >= 2
    P = sp.coo_matrix((g.normal(0, 0.05, keep.sum()), (i[keep], j[keep])), shape=(n, n)).tocsr()
    M = (synth.tridiag_toeplitz(n, 2.0, -1.0).to_scipy() + P + P.T).tocsr()
    M.sort_indices()
    A = synth.CSR(n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64),
                  M.diagonal().astype(np.float64))
    lam = np.linalg.eigvalsh(M.toarray())[:k]
    X0 = synth.gaussian_block(n, k, seed=7)
    r3 = oracle.lobpcg(A, A.diag, k, X0, tol=1e-9, maxiter=20000, precond=3)
    r1 = oracle.lobpcg(A, A.diag, k, X0, tol=1e-9, maxiter=20000, precond=1)
    assert r3.status == 0 and r1.status == 0
    assert np.max(rel_eig_err(r3.evals, lam)) <= 1e-10 and np.max(rel_eig_err(r1.evals, lam)) <= 1e-10
    assert 4 * r3.info["iterations"] <= 3 * r1.info["iterations"]


def test_lobpcg_tridiagonal_on_cfg1_matches_diagonal_eigenpairs():
    """cfg1 (n = 4096, seed 0): the tridiagonal and the diagonal preconditioner reach the
    same eigenvalues (a preconditioner changes the path, not the answer); 49 against 60
    iterations here."""
    a = synth.sparse_cfg1(n=4096, seed=0)
    X0 = synth.diag_guess(a.diag, 4, seed=0)
    r3 = oracle.lobpcg(a, a.diag, 4, X0, tol=1e-9, maxiter=2000, precond=3)
    r1 = oracle.lobpcg(a, a.diag, 4, X0, tol=1e-9, maxiter=2000, precond=1)
    assert r3.status == 0 and r1.status == 0
    assert np.max(rel_eig_err(r3.evals, r1.evals)) <= 1e-10
