"""Pins of the oracle's Algorithm 1 against closed forms, LAPACK and invariants."""
import warnings

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import oracle
import synth
from tests.util import cluster_angles, golden, max_subspace_angle, rel_eig_err


def test_diagonal_exact_start_exits_after_init():
    d = np.array([5.0, 0.5, 3.0, -1.0, 2.0, 7.0, 0.0, 4.0, 6.0, 1.5, 9.0, 8.0])
    A = np.diag(d)
    k = 3
    idx = np.argsort(d)[:k]
    X0 = np.asfortranarray(np.eye(12)[:, idx])
    r = oracle.lobpcg(A, d, k, X0)
    assert r.status == 0 and r.info["iterations"] == 0
    assert np.array_equal(r.evals, np.sort(d)[:k])
    assert np.all(r.resnorms == 0.0)
    assert np.array_equal(r.evecs, X0)


def test_diagonal_noisy_start_finds_smallest_entries():
    # Without a preconditioner: for a diagonal A the exact (D - theta)^-1 maps the residual
    # back onto x itself, so the diagonal preconditioner gives no new direction here.
    g = np.random.default_rng(0)
    n, k = 300, 5
    d = g.permutation(np.arange(n, dtype=float)) * 0.1
    A = np.diag(d)
    X0 = synth.gaussian_block(n, k, seed=2)
    r = oracle.lobpcg(A, d, k, X0, tol=1e-10, precond=0, maxiter=5000)
    assert r.status == 0
    assert np.max(np.abs(r.evals - np.arange(k) * 0.1)) <= 1e-14 * np.max(np.abs(d)) * k  # eps*||A|| scale
    for j in range(k):
        e = np.zeros(n)
        e[int(np.argmin(np.abs(d - 0.1 * j)))] = 1.0
        assert abs(abs(r.evecs[:, j] @ e) - 1.0) <= 1e-12


@pytest.mark.parametrize("n,a,b,k", [(60, 2.0, -1.0, 3), (200, 1.0, 0.3, 4)])
def test_tridiagonal_toeplitz_closed_form(n, a, b, k):
    """lambda_j = a + 2 b cos(j pi/(n+1)), v_j(i) ~ sin(i j pi/(n+1))."""
    A = synth.tridiag_toeplitz(n, a, b)
    j = np.arange(1, n + 1)
    lam = a + 2 * b * np.cos(j * np.pi / (n + 1))
    order = np.argsort(lam)[:k]
    i = np.arange(1, n + 1)[:, None]
    V = np.sin(i * j[order][None, :] * np.pi / (n + 1))
    V /= np.linalg.norm(V, axis=0)
    r = oracle.lobpcg(A, A.diag, k, synth.gaussian_block(n, k, seed=7), tol=1e-9, maxiter=20000)
    assert r.status == 0
    assert np.max(rel_eig_err(r.evals, lam[order])) <= 1e-12
    for jj in range(k):
        assert abs(abs(r.evecs[:, jj] @ V[:, jj]) - 1) <= 1e-9


@pytest.mark.parametrize("precond", [0, 1])
def test_dense_random_vs_lapack(precond):
    g = np.random.default_rng(11)
    n, k = 150, 5
    B = g.standard_normal((n, n))
    A = np.asfortranarray(0.5 * (B + B.T) + np.diag(np.linspace(0, 60, n)))
    w, v = np.linalg.eigh(A)
    r = oracle.lobpcg(A, np.diag(A).copy(), k, synth.gaussian_block(n, k, seed=1),
                      tol=1e-9, precond=precond, maxiter=5000)
    assert r.status == 0
    assert np.max(rel_eig_err(r.evals, w[:k])) <= 1e-12
    assert np.max(cluster_angles(w[:k], v[:, :k], r.evecs)) <= 1e-8
    assert np.max(r.resnorms) <= 1e-9 * 1.01


@pytest.fixture(scope="module")
def cfg1_run():
    a = synth.sparse_cfg1()
    x0 = synth.diag_guess(a.diag, 4, seed=0)
    r = oracle.lobpcg(a, a.diag, 4, x0, tol=1e-8)
    return a, r


def test_cfg1_matches_lapack_subset(cfg1_run):
    a, r = cfg1_run
    assert r.status == 0
    w, v = sla.eigh(a.to_scipy().toarray(), subset_by_index=[0, 5])
    assert np.max(rel_eig_err(r.evals, w[:4])) <= 1e-12
    assert np.max(cluster_angles(w[:4], v[:, :4], r.evecs)) <= 1e-7
    assert np.max(r.resnorms) <= 1e-8


def test_cfg1_invariants(cfg1_run):
    a, r = cfg1_run
    w = sla.eigh(a.to_scipy().toarray(), eigvals_only=True, subset_by_index=[0, 5])
    normA = spla.norm(a.to_scipy(), 1)
    H = r.hist_lambda
    # Ritz values per index never increase (V^[k] contains X^[k]) ...
    assert np.all(np.diff(H, axis=0) <= 1e-13 * normA)
    # ... and bound the true eigenvalues from above (Courant-Fischer)
    assert np.all(H >= w[None, :4] - 1e-13 * normA)
    # orthonormal output
    assert np.max(np.abs(r.evecs.T @ r.evecs - np.eye(4))) <= 1e-12
    # residual bounds on the error: |theta - lambda| <= ||r|| and <= ||r||^2 / gap
    gap = np.array([min(abs(w[j] - w[i]) for i in range(6) if i != j) for j in range(4)])
    assert np.all(np.abs(r.evals - w[:4]) <= r.resnorms + 1e-15)
    assert np.all(np.abs(r.evals - w[:4]) <= r.resnorms ** 2 / gap + 1e-14)
    # soft locking: the locked prefix is exactly the converged prefix of each step
    for row_res, mact in zip(r.hist_res, r.hist_mact):
        conv = row_res <= 1e-8
        prefix = int(np.argmin(conv)) if not conv.all() else len(conv)
        assert mact == len(conv) - prefix


def test_cfg1_paper_statistics(cfg1_run):
    """Sec. 3.2: at most 4 Cholesky-QR passes, ortho(X,Y) usually one or two passes (the
    printed values, tests/golden/paper_printed_values.json).  A claim about the paper's
    matrices, so a miss on this recipe warns; the loops must not hit their caps."""
    g = golden()
    _, r = cfg1_run
    if r.info["cholqr_passes_max"] > g["cholqr_passes_max"]["value"]:
        warnings.warn(f"Cholesky-QR passes {r.info['cholqr_passes_max']} > 4")
    if r.info["ortho_passes_max"] > g["ortho_against_passes_typical"]["value"] + 1:
        warnings.warn(f"ortho(X,Y) passes {r.info['ortho_passes_max']} > 3")
    assert r.info["cap_hits"] == 0 and r.info["svqb"] == 0


def test_matches_scipy_lobpcg_iteration_count_without_preconditioner():
    """Same method, independent implementation: unpreconditioned LOBPCG iteration counts agree."""
    a = synth.sparse_cfg1(n=1500, seed=5)
    x0 = synth.diag_guess(a.diag, 3, seed=5)
    r = oracle.lobpcg(a, a.diag, 3, x0, tol=1e-6, precond=0, maxiter=3000)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        w, _, h = spla.lobpcg(a.to_scipy(), x0.copy(), largest=False, tol=1e-6, maxiter=3000,
                              retResidualNormsHistory=True)
    assert r.status == 0
    assert np.max(rel_eig_err(r.evals, np.sort(w))) <= 1e-10
    assert abs(r.info["iterations"] - (len(h) - 1)) <= max(3, 0.1 * len(h))


def test_extra_block_columns():
    a = synth.sparse_cfg1(n=2000, seed=2)
    w = sla.eigh(a.to_scipy().toarray(), eigvals_only=True, subset_by_index=[0, 3])
    r = oracle.lobpcg(a, a.diag, 3, synth.diag_guess(a.diag, 6, seed=1), extra=3)
    assert r.status == 0 and r.evals.shape == (3,)
    assert np.max(rel_eig_err(r.evals, w[:3])) <= 1e-12


def test_tol_kind_rms_max():
    """tol_kind 1 is the paper's Full-CI criterion (Sec. 4.1): RMS residual <= 1e-9 and largest
    entry <= 1e-8 for tol = 1e-8 (values from tests/golden/paper_printed_values.json)."""
    g = golden()["fci_convergence"]
    a = synth.sparse_cfg1(n=2000, seed=2)
    r = oracle.lobpcg(a, a.diag, 2, synth.diag_guess(a.diag, 2, seed=1), tol=g["max"], tol_kind=1)
    assert r.status == 0
    n = a.n
    R = oracle.apply(a, r.evecs) - r.evecs * r.evals
    # criterion holds (up to the drift between maintained and fresh AX)
    assert np.all(np.linalg.norm(R, axis=0) / np.sqrt(n) <= g["rms"] * 1.5)
    assert np.max(np.abs(R)) <= g["max"] * 1.5


def test_maxiter_reports_noconv_with_best_result():
    a = synth.sparse_cfg1(n=2000, seed=2)
    r = oracle.lobpcg(a, a.diag, 2, synth.diag_guess(a.diag, 2, seed=1), maxiter=2)
    assert r.status == 4 and r.info["iterations"] == 2
    assert np.all(np.isfinite(r.evals)) and np.all(r.resnorms > 1e-8)


def test_invalid_arguments():
    A = np.eye(6)
    assert oracle.lobpcg(A, np.ones(6), 3, np.eye(6)[:, :3].copy(order="F")).status == 1  # 3m > n

