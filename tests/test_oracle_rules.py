"""Pins of the oracle's readings R6 (preconditioner guard), R14 (P only where x_j moved) and
R16 (drop what Algorithms 2-3 could not orthonormalise), each made to fire on an input where
the right answer is fixed by hand or by a dimension count."""
import numpy as np
import pytest

import oracle
import synth


# ------------------------------------------------------------------------------------ R6

def test_precondition_guard_sign_and_scale():
    """delta = d_i - lambda_j; |delta| < 1e-8 max(1, |lambda_j|) is replaced by
    sign(delta) 1e-8 max(1, |lambda_j|) with sign(0) = +1.  Expected denominators are
    written out by hand: column 0 has |lambda| < 1 (floor 1e-8), column 1 has lambda = 4
    (floor 4e-8), so a floor without the max(1, .) or with the wrong column's lambda, a
    negative sign(0) or a missing sign fails."""
    lam = np.array([0.25, 4.0])
    diag = np.array([0.25, 0.25 + 5e-9, 0.25 - 5e-9, 1.25, 4.0, 4.0 + 2e-8, 4.0 - 3e-8, 3.0])
    n = diag.size
    R = synth.gaussian_block(n, 2, seed=31)
    W = oracle.precondition(R, lam, diag, m_conv=0, m_act=2)
    den0 = np.array([1e-8, 1e-8, -1e-8, 1.0, 3.75, diag[5] - 0.25, diag[6] - 0.25, 2.75])
    den1 = np.array([0.25 - 4.0, diag[1] - 4.0, diag[2] - 4.0, 1.25 - 4.0, 4e-8, 4e-8, -4e-8, -1.0])
    assert np.array_equal(W[:, 0], R[:, 0] / den0)
    assert np.array_equal(W[:, 1], R[:, 1] / den1)
    # the active columns start at m_conv: column c of W uses lambda_{m_conv + c}
    W1 = oracle.precondition(R, lam, diag, m_conv=1, m_act=1)
    assert W1.shape == (n, 1) and np.array_equal(W1[:, 0], R[:, 1] / den1)
    # no preconditioner: W~ = R over the active columns
    assert np.array_equal(oracle.precondition(R, lam, diag, 0, 2, precond=0), R)


# ----------------------------------------------------------------------------------- R16

def _orthonormal(n, q, seed):
    return np.linalg.qr(synth.gaussian_block(n, q, seed))[0]


def test_drop_rule_threshold_sense_and_packing():
    """Overlaps between tau and sqrt(tau) are kept, above sqrt(tau) dropped; with the norm
    check a column whose norm is off by more than sqrt(tau) (or zero) is dropped; kept
    columns come back bit for bit, packed in their original order."""
    n, q = 50, 3
    Q = _orthonormal(n, q + 7, seed=32)
    Y, U = Q[:, :q], Q[:, q:]  # U: orthonormal, orthogonal to Y
    cols = [
        U[:, 0],                                         # 0 keep
        np.sqrt(1 - 1e-18) * U[:, 1] + 1e-9 * Y[:, 0],   # 1 overlap 1e-9: keep (tau < 1e-9 < sqrt(tau))
        np.sqrt(1 - 1e-12) * U[:, 2] + 1e-6 * Y[:, 1],   # 2 overlap 1e-6: drop
        (1 + 1e-6) * U[:, 3],                            # 3 norm off by 1e-6: drop with the norm check
        (1 + 1e-9) * U[:, 4],                            # 4 norm off by 1e-9: keep
        np.zeros(n),                                     # 5 zero: drop with the norm check
        U[:, 5],                                         # 6 keep
    ]
    W = np.asfortranarray(np.stack(cols, axis=1))
    kept = oracle.drop_unorthogonal_columns(W, Y, tau=1e-14, check_norm=True)
    assert kept.shape[1] == 4 and np.array_equal(kept, W[:, [0, 1, 4, 6]])
    kept = oracle.drop_unorthogonal_columns(W, Y, tau=1e-14, check_norm=False)
    assert kept.shape[1] == 6 and np.array_equal(kept, W[:, [0, 1, 3, 4, 5, 6]])
    # without Y only the norms are tested
    kept = oracle.drop_unorthogonal_columns(W, None, tau=1e-14, check_norm=True)
    assert np.array_equal(kept, W[:, [0, 1, 2, 4, 6]])


def test_exhausted_complement_hits_the_cap_and_drops_the_last_column():
    """p columns against q orthonormal ones in R^(q+p-1): only p-1 directions are
    orthogonal to Y, so Algorithm 3 cannot succeed and stops at its cap (the situation of
    u_p in R^s after a column unlocks).  R16 must then drop exactly one column, the last
    in Cholesky order; the kept ones are the QR factor of the projected first p-1
    columns (up to signs), orthonormal, orthogonal to Y, and with Y they span the whole
    space, so no direction of the input is lost."""
    q, p = 5, 5
    n = q + p - 1
    Y = _orthonormal(n, q, seed=33)
    Xt = synth.gaussian_block(n, p, seed=34)
    X, st = oracle.ortho_against(Xt, Y, tau=1e-14, cap=6, cap2=4)
    assert st["cap_hits"] >= 1
    kept = oracle.drop_unorthogonal_columns(X, Y, tau=1e-14, check_norm=True)
    assert kept.shape[1] == p - 1
    assert np.max(np.abs(kept.T @ kept - np.eye(p - 1))) <= 1e-12
    assert np.max(np.abs(Y.T @ kept)) <= 1e-12
    Qref = np.linalg.qr(Xt[:, : p - 1] - Y @ (Y.T @ Xt[:, : p - 1]))[0]
    assert np.max(np.abs(np.abs(Qref.T @ kept) - np.eye(p - 1))) <= 1e-10
    B = np.hstack([Y, kept])
    coef = np.linalg.lstsq(B, Xt, rcond=None)[0]
    assert np.max(np.abs(B @ coef - Xt)) <= 1e-12 * np.max(np.abs(Xt))


def test_no_cap_no_drop():
    """With room for every column Algorithm 3 converges and R16 never fires."""
    n, q, p = 400, 6, 5
    Y = _orthonormal(n, q, seed=35)
    Xt = synth.gaussian_block(n, p, seed=36)
    Xt[:, 2] = Y @ np.arange(1.0, q + 1) + 1e-17 * Xt[:, 2]  # a column inside span(Y)
    X, st = oracle.ortho_against(Xt, Y)
    assert st["cap_hits"] == 0
    assert np.max(np.abs(X.T @ X - np.eye(p))) <= 1e-14 * 4
    assert np.max(np.abs(Y.T @ X)) <= 1e-14


# ------------------------------------------------------------------------- R14 with R16

def _exact_pair_problem(n=20, seed=37):
    """Diagonal A = diag(1..n); x_1 = e_0 + noise (noise zero at row 1) and x_2 = e_1 exactly.
    x_2 is an exact eigenvector behind an unconverged x_1, so it stays active; every
    coupling with it is exactly zero, its Jacobi column stays a unit vector (u~_p = 0) and
    its residual, hence its W~ column, is exactly zero.  Solved without a preconditioner:
    for a diagonal A the diagonal one is exact, T r_1 is parallel to x_1 and its projection
    is rounding noise, a second degeneracy that would hide this one."""
    d = np.arange(1.0, n + 1)
    x1 = np.zeros(n)
    x1[0] = 1.0
    noise = 1e-3 * synth.gaussian_block(n, 1, seed=seed)[:, 0]
    noise[1] = 0.0
    X0 = np.asfortranarray(np.stack([x1 + noise, np.eye(n)[:, 1]], axis=1))
    return np.diag(d), d, X0


def test_exact_active_pair_drops_its_p_and_w_columns():
    A, d, X0 = _exact_pair_problem()
    r = oracle.lobpcg(A, d, 2, X0, tol=1e-10, maxiter=200, precond=0)
    assert r.status == 0
    assert np.max(np.abs(r.evals - [1.0, 2.0])) <= 1e-14
    assert np.all(np.isfinite(r.resnorms)) and np.max(r.resnorms) <= 1e-10
    assert abs(abs(r.evecs[0, 0]) - 1.0) <= 1e-12 and abs(r.evecs[1, 1]) == 1.0
    # while both pairs are active: W has one column (the zero W~ column is dropped, R16)
    # and, from the second step on, P has one column (x_2 did not move, R14)
    assert r.hist_mact[0] == 2
    assert np.all(r.hist_wcols[1:] == 1)
    assert np.all(r.hist_pcols[2:] == 1) and r.hist_pcols[1] == 0
    # W is built after every step but the last, P after every step but the first and last
    rows = len(r.hist_mact)
    assert r.info["w_dropped"] == rows - 1 and r.info["p_dropped"] == rows - 2


def test_cfg1_run_never_drops():
    a = synth.sparse_cfg1()
    x0 = synth.diag_guess(a.diag, 4, seed=0)
    r = oracle.lobpcg(a, a.diag, 4, x0, tol=1e-8)
    assert r.status == 0 and r.info["cap_hits"] == 0
    assert r.info["w_dropped"] == 0 and r.info["p_dropped"] == 0
    # the basis has its full width at every step: W = m_act columns, P = m_act of the previous step
    assert np.all(r.hist_wcols[1:] == r.hist_mact[:-1])
    assert r.hist_pcols[1] == 0 and np.all(r.hist_pcols[2:] == r.hist_mact[1:-1])


# ------------------------------------------------------------- R17, R18 (Sec. 3.2 trims)

def test_recheck_skip_only_after_a_well_conditioned_pass():
    """R17: the re-check Gram of Algorithm 2 is skipped only after an unshifted pass with
    ||F||_F <= 1/2 (F = scaled overlap - I), where ||L^-T||^2 <= 2 and the new vectors are
    orthonormal to the Gram's rounding.  A nearly orthonormal block (||F||_F ~ 0.2) needs
    one pass and no re-check; an ill-conditioned one (cond ~ 1e5) gets its re-check after
    the first pass and skips it after the second.  The output equals the printed
    algorithm's bit for bit (the skipped test would have passed) and is orthonormal to tau
    checked in numpy."""
    n, p = 600, 6
    good = synth.gaussian_block(n, p, seed=40)
    bad = good.copy()
    bad[:, 3] = bad[:, 1] + 1e-5 * bad[:, 3]  # nearly dependent columns
    for X, grams_trim, grams_plain in ((good, 1, 2), (bad, 2, 3)):
        Q0, s0 = oracle.ortho(X, trim=False)
        Q1, s1 = oracle.ortho(X, trim=True)
        assert np.array_equal(Q0, Q1) and s0["passes"] == s1["passes"]
        assert s1["grams"] == grams_trim and s0["grams"] == grams_plain
        assert s1["skipped_recheck"] == 1 and s0["skipped_recheck"] == 0
        assert np.max(np.abs(Q1.T @ Q1 - np.eye(p))) <= 1e-14


def test_growth_factor_exit_only_when_little_was_projected_out():
    """R18: Algorithm 3 skips its test Gram Y^T X when eps sqrt(q) g <= tau, g the growth
    factor ||x~_j|| / ||x_proj,j|| * ||L^-T|| of the pass.  A block with a small component
    in span(Y) has g ~ 1: one pass, no test Gram, same output as the printed algorithm and
    orthogonal to Y to tau (numpy).  A block almost inside span(Y) (g ~ 1e6) keeps the
    test after its first pass and takes a second one, whose growth is ~1 again (its test
    is skipped)."""
    n, q, p = 600, 8, 5
    Y = _orthonormal(n, q, seed=41)
    Xs = synth.gaussian_block(n, p, seed=42)
    near = Y @ synth.gaussian_block(q, p, seed=43) + 1e-6 * Xs
    for Xt, passes, skipped in ((Xs, 1, 1), (near, 2, 1)):
        Q0, s0 = oracle.ortho_against(Xt, Y, trim=False)
        Q1, s1 = oracle.ortho_against(Xt, Y, trim=True)
        assert s1["passes"] == passes and s1["skipped_test"] == skipped
        assert np.array_equal(Q0, Q1) and s0["passes"] == passes
        assert s0["grams"] - s1["grams"] == skipped + s1["skipped_recheck"]
        assert np.max(np.abs(Y.T @ Q1)) <= 1e-14
        assert np.max(np.abs(Q1.T @ Q1 - np.eye(p))) <= 1e-14


@pytest.mark.parametrize("case", ["cfg1", "ci", "dense"])
def test_trimmed_lobpcg_is_the_printed_one_with_fewer_grams(case):
    """On these runs every skipped Gram's test would have passed, so the trimmed method
    reproduces the printed Algorithms 2-3 bit for bit with 15-30% fewer orthogonalisation
    Grams (the paper's claim of <= 4 Cholesky-QR passes and ~2 ortho(X, Y) passes holds)."""
    if case == "cfg1":
        a = synth.sparse_cfg1()
        A, d, k, extra, x0 = a, a.diag, 4, 0, synth.diag_guess(a.diag, 4, seed=0)
    elif case == "ci":
        a = synth.sparse_ci(n=20_011, seed=2105)
        A, d, k, extra, x0 = a, a.diag, 6, 2, synth.diag_guess(a.diag, 8, seed=2105, noise=0.0)
    else:
        A, d = synth.dense_casscf(n=1024, seed=2, rank=64)
        k, extra, x0 = 4, 0, synth.diag_guess(d, 4, seed=2)
    r0 = oracle.lobpcg(A, d, k, x0, extra=extra, tol=1e-8, maxiter=3000, trim=False)
    r1 = oracle.lobpcg(A, d, k, x0, extra=extra, tol=1e-8, maxiter=3000, trim=True)
    assert r0.status == 0 and r1.status == 0
    assert np.array_equal(r0.evals, r1.evals) and np.array_equal(r0.evecs, r1.evecs)
    saved = r1.info["skipped_recheck"] + r1.info["skipped_test"]
    assert r0.info["ortho_grams"] - r1.info["ortho_grams"] == saved
    assert 0.15 * r0.info["ortho_grams"] <= saved
    assert r1.info["cholqr_passes_max"] <= 4 and r1.info["ortho_passes_max"] <= 3
