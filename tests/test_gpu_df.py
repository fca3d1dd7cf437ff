"""Double-float FP64 products (the refinement phase's Gram, block update and CSR product on
the FP32 pipes) against the CPU oracle's FP64 arithmetic.

Bound, per entry: |C - C_ref| <= (8 + k) 2^-47 sum|terms|, k the number of terms summed in
double-float before an FP64 add.  A split x = hi + lo keeps x to 2^-47 |x| and a product of
split pairs errs by a few 2^-48 (together <= 8 2^-47); each compensated addition (TwoSum
then Fast2Sum, a double-word plus float addition) errs by at most 2u^2 = 2^-47 of its
result (Joldes, Muller and Popescu, 2017), and every partial sum is bounded by
sum|terms|.  Still five orders of magnitude below FP32's 2^-24.  On small integers every
split, product and sum is exact, so the Gram must equal the integer Gram bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import cuda, dev
from tests.util import cluster_angles, rel_eig_err

pytestmark = pytest.mark.gpu

def bound(k):
    return (8 + k) * 2.0 ** -47


# terms per double-float sum: the Gram flushes a thread's sums to FP64 every ~128 rows
GRAM_K, BOUND = 128, bound(128)


def _rowmajor(torch, M, ld):
    n, w = M.shape
    buf = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
    buf[:, :w] = torch.from_numpy(np.ascontiguousarray(M)).cuda()
    return buf[:, :w]


@pytest.mark.parametrize("n,p,q,spread", [(1, 1, 1, 0), (37, 3, 5, 0), (100_003, 21, 21, 0), (200_003, 63, 63, 0),
                                          (50_001, 96, 96, 0), (70_001, 42, 21, 10)])
def test_gram_df_matches_oracle(n, p, q, spread):
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    X = synth.gaussian_block(n, p, seed=n + p)
    Y = synth.gaussian_block(n, q, seed=n + q + 1)
    if spread:
        # row scales 10^U(-spread, spread): products over 2 * spread decades in one sum
        g = np.random.default_rng(n)
        X *= (10.0 ** g.uniform(-spread, spread, n))[:, None]
        Y *= (10.0 ** g.uniform(-spread, spread, n))[:, None]
    ld = max(p, q) + (max(p, q) & 1)
    Xd, Yd = _rowmajor(torch, X, ld), _rowmajor(torch, Y, ld)
    got = lb.gram_df(Xd, Yd).cpu().numpy()
    ref = oracle.gram(X, Y)
    scale = np.abs(X).T @ np.abs(Y)
    err = np.abs(got - ref)
    assert np.all(err <= BOUND * scale + 1e-300), float(np.max(err / scale))
    # and the FP64 FMA kernel agrees to the same bound
    d64 = lb.gram(Xd, Yd).cpu().numpy()
    assert np.all(np.abs(got - d64) <= 2 * BOUND * scale + 1e-300)


def test_gram_df_exact_on_small_integers():
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    g = np.random.default_rng(3)
    n, p = 30_011, 24
    X = g.integers(-2048, 2049, size=(n, p)).astype(np.float64)
    Y = g.integers(-2048, 2049, size=(n, p)).astype(np.float64)
    got = lb.gram_df(dev(torch, X), dev(torch, Y)).cpu().numpy()
    exact = (X.astype(np.int64).T @ Y.astype(np.int64)).astype(np.float64)  # |sums| < 2^37: exact in FP64
    assert np.array_equal(got, exact)


@pytest.mark.parametrize("mode", ["pair_norm", "base_inplace", "right_inplace", "plain", "plain_odd_ld",
                                  "pair_norm_ragged"])
def test_update_f64_df_matches_oracle(mode):
    """X = base + alpha [V_g] U in double-float against the oracle's FP64 product (V U as a
    Gram of V^T and U over the s rows), to (8 + s + 1) 2^-47 (|V| |U|) (+ |base|).  Even row
    strides take the kernel that stages the next slab asynchronously; an odd stride
    (plain_odd_ld) takes the synchronous one; ragged segment widths and a row count that is
    not a multiple of the slab exercise the padding and the last slab."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    n, ws, q = 90_001, [21, 21, 21], 21
    if mode == "right_inplace":
        ws, q = [21], 21
    if mode == "pair_norm_ragged":
        n, ws, q = 77_777, [7, 22, 13], 9
    s = sum(ws)
    ld = 23 if mode == "plain_odd_ld" else 24
    Vs = [synth.gaussian_block(n, w, seed=500 + i) for i, w in enumerate(ws)]
    AVs = [synth.gaussian_block(n, w, seed=600 + i) for i, w in enumerate(ws)]
    U = synth.gaussian_block(s, q, seed=17) / np.sqrt(s)
    Vd = [_rowmajor(torch, M, ld) for M in Vs]
    AVd = [_rowmajor(torch, M, ld) for M in AVs]
    Ud = torch.from_numpy(U).cuda()
    Vcat, AVcat = np.hstack(Vs), np.hstack(AVs)
    ref = oracle.gram(Vcat.T.copy(), U)
    BOUND = bound(s + 1)  # s products and the base
    tol = BOUND * (np.abs(Vcat) @ np.abs(U)) + 1e-300
    if mode.startswith("pair_norm"):
        lam = np.linspace(-1.0, 2.0, q)
        X, AX, rn = lb.update_f64_df(Vd, Ud, AV=AVd, lam=torch.from_numpy(lam).cuda(), resnorm=True)
        Xh, AXh = X.cpu().numpy(), AX.cpu().numpy()
        assert np.all(np.abs(Xh - ref) <= tol)
        aref = oracle.gram(AVcat.T.copy(), U)
        assert np.all(np.abs(AXh - aref) <= BOUND * (np.abs(AVcat) @ np.abs(U)) + 1e-300)
        R = AXh - Xh * lam[None, :]
        rn_ref = np.sqrt(np.sum(R * R, axis=0))
        assert np.all(np.abs(rn - rn_ref) <= 1e-13 * rn_ref)
    elif mode == "base_inplace":
        W0 = synth.gaussian_block(n, q, seed=19)
        W = _rowmajor(torch, W0, ld)
        out = lb.update_f64_df(Vd, Ud, alpha=-1.0, base=W, X=W)
        assert out.data_ptr() == W.data_ptr()
        assert np.all(np.abs(W.cpu().numpy() - (W0 - ref)) <= tol + BOUND * np.abs(W0))
    elif mode == "right_inplace":
        lb.update_f64_df(Vd, Ud, X=Vd[0][:, :q])
        assert np.all(np.abs(Vd[0][:, :q].cpu().numpy() - ref) <= tol)
    else:
        X = lb.update_f64_df(Vd, Ud)
        assert np.all(np.abs(X.cpu().numpy() - ref) <= tol)


def test_fp64_solves_with_df_products_match_oracle():
    """Every FP64 Gram and update of the solve in double-float (df_products=1): the
    eigenpairs still match the oracle at the FP64 path's bars (1e-10 relative eigenvalues,
    1e-7 principal angles) on a CI-like banded matrix and on a dense ill-conditioned one."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    a = synth.sparse_ci(n=60_001, seed=5)
    k = 6
    x0 = synth.diag_guess(a.diag, k, seed=5, noise=0.0)
    ref = oracle.lobpcg(a, a.diag, k, x0, tol=1e-8)
    s = lb.Solver(**lb.upload_csr(a), df_products=1)
    res = s.solve(k, 1e-8, X0=torch.from_numpy(x0).cuda())
    s.close()
    assert ref.status == 0 and res.status == 0 and res.info["df_products"] == 1
    assert np.max(rel_eig_err(res.evals, ref.evals)) <= 1e-10
    assert np.max(cluster_angles(ref.evals, ref.evecs, res.evecs.cpu().numpy())) <= 1e-7
    assert np.max(res.resnorms) <= 1e-8
    A, d = synth.dense_casscf(n=1024, seed=2, rank=64)
    x0 = synth.diag_guess(d, 4, seed=2)
    ref = oracle.lobpcg(A, d, 4, x0, tol=1e-8, maxiter=3000)
    s = lb.Solver(diag=dev(torch, d), dense=torch.from_numpy(A).cuda(), df_products=1, maxiter=3000)
    res = s.solve(4, 1e-8, X0=torch.from_numpy(x0).cuda())
    s.close()
    assert ref.status == 0 and res.status == 0
    assert np.max(rel_eig_err(res.evals, ref.evals)) <= 1e-10
    assert np.max(cluster_angles(ref.evals, ref.evecs, res.evecs.cpu().numpy())) <= 1e-7


@pytest.mark.parametrize("n,p", [(5003, 1), (40_009, 8), (60_001, 21), (30_011, 32)])
def test_spmm_df_matches_oracle(n, p):
    """Y = A X in double-float against the oracle's FP64 product, element by element, on a
    CI-like banded matrix (empty and long rows included by the recipe's ends)."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    a = synth.sparse_ci(n=n, seed=n)
    X = synth.gaussian_block(n, p, seed=p)
    ld = p + (p & 1)
    Xd = _rowmajor(torch, X, ld)
    Yd = _rowmajor(torch, np.zeros((n, p)), ld)
    t = lb.upload_csr(a)
    lb.spmm_csr_df(t["row_ptr"], t["col_idx"], t["val"], Xd, Yd)
    got = Yd.cpu().numpy()
    ref = oracle.apply(a, X)
    absA = a.to_scipy().copy()
    absA.data = np.abs(absA.data)
    scale = absA @ np.abs(X)
    ratio = np.abs(got - ref) / (scale + 1e-300)
    i, j = np.unravel_index(np.argmax(ratio), ratio.shape)
    kmax = int(np.max(np.diff(a.row_ptr)))  # terms of the longest row
    assert ratio[i, j] <= bound(kmax), (i, j, ratio[i, j], got[i, j], ref[i, j], scale[i, j])
