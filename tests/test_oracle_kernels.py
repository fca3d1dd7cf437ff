"""Pins of the oracle's building blocks against library routines and closed forms.

Each check compares the oracle with something other than itself: numpy/scipy LAPACK
routines, closed-form results, or mathematical invariants.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from tests.util import max_subspace_angle


def sym(s, seed):
    g = np.random.default_rng(seed)
    a = g.standard_normal((s, s))
    return 0.5 * (a + a.T)


@pytest.mark.parametrize("s", [1, 2, 3, 7, 12, 48, 96])
def test_jacobi_matches_lapack(s):
    a = sym(s, s)
    lam, U, sweeps = oracle.jacobi_eig(a)
    ref = np.linalg.eigvalsh(a)
    nrm = np.linalg.norm(a)
    assert sweeps >= 0
    assert np.max(np.abs(lam - ref)) <= 1e-13 * max(nrm, 1.0)
    assert np.max(np.abs(U.T @ U - np.eye(s))) <= 1e-13 * s
    assert np.linalg.norm(a @ U - U * lam) <= 1e-13 * max(nrm, 1.0) * s
    assert np.all(np.diff(lam) >= 0)


def test_jacobi_2x2_closed_form():
    a, b, c = 0.3, -1.7, 2.5
    lam, U, _ = oracle.jacobi_eig(np.array([[a, b], [b, c]]))
    mid, rad = 0.5 * (a + c), np.hypot(0.5 * (a - c), b)
    assert np.allclose(lam, [mid - rad, mid + rad], rtol=0, atol=1e-15 * 4)
    # eigenvector of the smaller eigenvalue is orthogonal to (b, lam0 - a)
    v = U[:, 0]
    assert abs(v @ np.array([lam[0] - a, -b])) / np.hypot(lam[0] - a, b) < 1e-14 or abs(
        (a - lam[0]) * v[0] + b * v[1]) < 1e-14


def test_jacobi_diagonal_and_ties():
    lam, U, sweeps = oracle.jacobi_eig(np.diag([1.0, 1.0, 0.0]))
    assert sweeps == 0
    assert list(lam) == [0.0, 1.0, 1.0]
    # stable order: the eigenvalue 0 is index 2, then the tied ones in index order
    assert np.array_equal(U, np.eye(3)[:, [2, 0, 1]])


def test_cholesky_matches_lapack_and_reports_failure():
    g = np.random.default_rng(1)
    B = g.standard_normal((20, 9))
    M = B.T @ B
    L, fail = oracle.cholesky(M)
    assert fail == 0
    assert np.max(np.abs(L - np.linalg.cholesky(M))) <= 1e-13 * np.max(np.abs(M))
    _, fail = oracle.cholesky(np.diag([1.0, 2.0, -1.0, 4.0]))
    assert fail == 3
    _, fail = oracle.cholesky(np.array([[1.0, 1.0], [1.0, 1.0]]))
    assert fail == 2  # exactly singular: pivot 0


@pytest.mark.parametrize("n,p,q", [(1, 1, 1), (37, 3, 5), (1000, 7, 7), (4099, 16, 48)])
def test_gram_matches_matmul(n, p, q):
    g = np.random.default_rng(n)
    X = np.asfortranarray(g.standard_normal((n, p)))
    Y = np.asfortranarray(g.standard_normal((n, q)))
    C = oracle.gram(X, Y)
    assert np.max(np.abs(C - X.T @ Y)) <= 1e-13 * np.sqrt(n) * 4


def test_gram_as_block_product_with_many_outputs():
    """The block product V U (n x s times s x q) written as the Gram (V^T)^T U over s rows,
    the form the FP32 update parity test uses: checked element by element against integer
    arithmetic (exact) and against a float product (every entry of the n x q result, with
    n far above the Gram's usual widths)."""
    g = np.random.default_rng(5)
    n, s, q = 20_011, 63, 21
    # small integers: every product and sum is exact in FP64, so the result must be exact
    Vi = g.integers(-64, 65, size=(n, s))
    Ui = g.integers(-64, 65, size=(s, q))
    C = oracle.gram(Vi.T.astype(np.float64).copy(), Ui.astype(np.float64))
    assert C.shape == (n, q)
    assert np.array_equal(C, (Vi @ Ui).astype(np.float64))
    # general values: within the pairwise-summation bound of the exact product
    V = g.standard_normal((n, s))
    U = g.standard_normal((s, q))
    C = oracle.gram(V.T.copy(), U)
    scale = np.abs(V) @ np.abs(U)
    assert np.all(np.abs(C - V @ U) <= 8 * np.finfo(float).eps * scale)


def test_apply_matches_scipy_and_dense():
    a = synth.sparse_cfg1(n=600, seed=3)
    X = synth.gaussian_block(600, 5, seed=1)
    ref = a.to_scipy() @ X
    assert np.max(np.abs(oracle.apply(a, X) - ref)) <= 1e-14
    d = synth.dense_from_csr(a)
    assert np.max(np.abs(oracle.apply(d, X) - ref)) <= 1e-14


def _qr_pos(X):
    q, r = np.linalg.qr(X)
    s = np.sign(np.diag(r))
    s[s == 0] = 1
    return q * s


def test_ortho_equals_householder_q():
    """Cholesky-QR gives the unique QR factor with positive diagonal R = L^T."""
    g = np.random.default_rng(2)
    X = np.asfortranarray(g.standard_normal((2000, 10)) @ np.diag(10.0 ** np.arange(10)))
    Q, st = oracle.ortho(X)
    assert np.max(np.abs(Q.T @ Q - np.eye(10))) <= 1e-14
    assert np.max(np.abs(Q - _qr_pos(X))) <= 1e-10
    assert 1 <= st["passes"] <= 4 and st["shifts"] == 0


def test_ortho_shifted_path_on_ill_conditioned_block():
    """cond(X) ~ 1e12 > 1e8: plain Cholesky of X^T X fails and the shift must rescue it."""
    g = np.random.default_rng(3)
    U, _ = np.linalg.qr(g.standard_normal((3000, 8)))
    Vt, _ = np.linalg.qr(g.standard_normal((8, 8)))
    X = np.asfortranarray(U @ np.diag(np.logspace(0, -12, 8)) @ Vt)
    Q, st = oracle.ortho(X)
    assert st["shifts"] >= 1
    assert np.max(np.abs(Q.T @ Q - np.eye(8))) <= 1e-14
    # same column space as X (the directions are resolved to ~ eps * cond)
    assert max_subspace_angle(Q, U) < 1e-3
    # paper's statistic (Sec. 3.2): a failed, a shifted, then at most two plain passes
    assert st["passes"] <= 4


def test_svqb_orthonormalises_and_keeps_span():
    g = np.random.default_rng(4)
    X = np.asfortranarray(g.standard_normal((500, 6)) * np.array([1, 1e-3, 1e3, 1, 5, 1e-6]))
    Q = oracle.svqb(X)
    assert np.max(np.abs(Q.T @ Q - np.eye(6))) <= 1e-9
    assert max_subspace_angle(Q, X) < 1e-8


def test_ortho_against_orthogonality_and_span():
    g = np.random.default_rng(5)
    Y, _ = np.linalg.qr(g.standard_normal((3000, 12)))
    Y = np.asfortranarray(Y)
    # X~ almost inside span(Y): the projected part is 1e-9 relative
    Xt = np.asfortranarray(Y @ g.standard_normal((12, 5)) + 1e-9 * g.standard_normal((3000, 5)))
    Q, st = oracle.ortho_against(Xt, Y)
    assert np.max(np.abs(Y.T @ Q)) <= 1e-14
    assert np.max(np.abs(Q.T @ Q - np.eye(5))) <= 1e-14
    # span(Y, Q) contains X~
    B = np.hstack([Y, Q])
    res = Xt - B @ np.linalg.lstsq(B, Xt, rcond=None)[0]
    assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(Xt)
    # one projection pass leaves eps/1e-9 ~ 1e-7 overlap: a second pass is needed (Sec. 3.2)
    assert st["passes"] >= 2 and st["passes"] <= 4


def test_ortho_against_already_orthogonal_still_normalises():
    """Reading R5: the body runs at least once, so X~ orthogonal to Y still gets normalised."""
    Y = np.asfortranarray(np.eye(10)[:, :3])
    Xt = np.asfortranarray(np.eye(10)[:, 3:6] * 7.0)
    Q, st = oracle.ortho_against(Xt, Y)
    assert np.allclose(Q, np.eye(10)[:, 3:6], atol=1e-15)
    assert st["passes"] == 1
