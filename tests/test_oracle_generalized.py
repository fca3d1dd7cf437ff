"""Pins of the oracle's generalised LOBPCG (A x = lambda B x, Sec. 3.3) against LAPACK's
generalised symmetric eigensolver, closed forms and the invariants of a B-orthonormal basis."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import synth
from tests.util import max_subspace_angle, rel_eig_err


def _spd(n, seed, cond=10.0):
    g = np.random.default_rng(seed)
    q, _ = np.linalg.qr(g.standard_normal((n, n)))
    d = np.geomspace(1.0, cond, n)
    return np.asfortranarray((q * d) @ q.T)


def test_identity_mass_reproduces_the_standard_method():
    """With B = I every step of the generalised method reduces to Algorithm 1: the same
    iterations, eigenvalues to rounding, eigenvectors to the residual level (the rounding of
    the extra orthonormalisation of (B X, B P) = (X, P) differs)."""
    a = synth.sparse_cfg1(n=2000, seed=2)
    eye = synth.tridiag_toeplitz(2000, 1.0, 0.0)
    x0 = synth.diag_guess(a.diag, 3, seed=1)
    r0 = oracle.lobpcg(a, a.diag, 3, x0, tol=1e-8)
    r1 = oracle.lobpcg_gen(a, eye, a.diag, eye.diag, 3, x0, tol=1e-8)
    assert r0.status == 0 and r1.status == 0
    assert r0.info["iterations"] == r1.info["iterations"]
    assert np.max(rel_eig_err(r1.evals, r0.evals)) <= 1e-15
    for j in range(3):
        assert max_subspace_angle(r0.evecs[:, j:j + 1], r1.evecs[:, j:j + 1]) <= 1e-9


def test_diagonal_pair_closed_form():
    """A = diag(a), B = diag(b): lambda_i = a_i / b_i, eigenvectors unit vectors scaled to
    x^T B x = 1 (x = e_i / sqrt(b_i))."""
    n, k = 60, 4
    g = np.random.default_rng(4)
    av = g.uniform(1.0, 10.0, n)
    bv = g.uniform(0.5, 3.0, n)
    A, B = np.diag(av), np.diag(bv)
    lam = av / bv
    order = np.argsort(lam)[:k]
    r = oracle.lobpcg_gen(A, B, av, bv, k, synth.gaussian_block(n, k, seed=5), tol=1e-10, precond=0,
                          maxiter=5000)
    assert r.status == 0
    assert np.max(rel_eig_err(r.evals, lam[order])) <= 1e-13
    for j, i in enumerate(order):
        assert abs(abs(r.evecs[i, j]) - 1.0 / np.sqrt(bv[i])) <= 1e-10


@pytest.mark.parametrize("cond,precond", [(10.0, 1), (1e4, 1), (10.0, 0)])
def test_dense_pair_against_lapack(cond, precond):
    """Random symmetric A and SPD B (condition up to 1e4, the paper's point that the
    re-use of B W^ holds even for an ill-conditioned B): eigenvalues against LAPACK's
    generalised eigh, eigenvectors by angle, x^T B x = I, residuals at tol."""
    n, k = 200, 4
    g = np.random.default_rng(7)
    M = g.standard_normal((n, n))
    A = np.asfortranarray(0.5 * (M + M.T) + np.diag(np.linspace(0, 40, n)))
    B = _spd(n, 8, cond)
    w, v = sla.eigh(A, B)
    r = oracle.lobpcg_gen(A, B, np.diag(A).copy(), np.diag(B).copy(), k, synth.gaussian_block(n, k, seed=3),
                          tol=1e-9, maxiter=5000, precond=precond)
    assert r.status == 0
    assert np.max(rel_eig_err(r.evals, w[:k])) <= 1e-11
    for j in range(k):
        assert max_subspace_angle(v[:, j:j + 1], r.evecs[:, j:j + 1]) <= 1e-7
    assert np.max(np.abs(r.evecs.T @ B @ r.evecs - np.eye(k))) <= 1e-12
    R = A @ r.evecs - (B @ r.evecs) * r.evals
    assert np.allclose(np.linalg.norm(R, axis=0), r.resnorms, rtol=1e-6, atol=1e-14)
    assert np.max(r.resnorms) <= 1e-9
    # Ritz values of every step bound the true eigenvalues from above
    assert np.all(r.hist_lambda >= w[None, :k] - 1e-12 * np.max(np.abs(w)))


def test_sparse_pair_against_lapack():
    """CSR A (cfg1 recipe) with a sparse SPD mass matrix B = I + 0.1 * tridiag(1, -0.5)."""
    n, k = 1500, 3
    a = synth.sparse_cfg1(n=n, seed=6)
    b = synth.tridiag_toeplitz(n, 1.0, -0.05)
    x0 = synth.diag_guess(a.diag, k, seed=6)
    r = oracle.lobpcg_gen(a, b, a.diag, b.diag, k, x0, tol=1e-9, maxiter=3000)
    assert r.status == 0
    w = sla.eigh(a.to_scipy().toarray(), b.to_scipy().toarray(), eigvals_only=True, subset_by_index=[0, k])
    assert np.max(rel_eig_err(r.evals, w[:k])) <= 1e-12
