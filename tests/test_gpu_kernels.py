"""GPU building blocks (through the C ABI) against the CPU oracle, element by element."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import cuda, dev
from tests.util import max_subspace_angle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,p", [(1, 1), (97, 3), (4096, 4), (20011, 16), (5003, 32), (3001, 7)])
def test_spmm_csr_matches_oracle(n, p):
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    a = synth.sparse_cfg1(n=max(n, 3), seed=n) if n >= 3 else synth.tridiag_toeplitz(3, 1.0, 0.5)
    n = a.n
    X = synth.gaussian_block(n, p, seed=1)
    t = lb.upload_csr(a)
    Y = lb.spmm_csr(t["row_ptr"], t["col_idx"], t["val"], dev(torch, X)).cpu().numpy()
    ref = oracle.apply(a, X)
    scale = np.abs(a.to_scipy()) @ np.abs(X)
    assert np.all(np.abs(Y - ref) <= 4 * np.finfo(float).eps * 64 * (scale + 1e-300))


def test_spmm_csr_ci_band_matrix_ragged_tail():
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    a = synth.sparse_ci(n=50_001, seed=4)
    X = synth.gaussian_block(a.n, 16, seed=2)
    t = lb.upload_csr(a)
    Y = lb.spmm_csr(t["row_ptr"], t["col_idx"], t["val"], dev(torch, X)).cpu().numpy()
    ref = oracle.apply(a, X)
    scale = np.abs(a.to_scipy()) @ np.abs(X)
    assert np.all(np.abs(Y - ref) <= 4 * np.finfo(float).eps * 80 * scale)


@pytest.mark.parametrize("n,p", [(1, 1), (300, 4), (1031, 8), (2048, 13), (8193, 21), (500, 32), (700, 9), (1500, 2), (999, 3)])
def test_spmm_dense_matches_oracle(n, p):
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    g = np.random.default_rng(n)
    B = g.standard_normal((n, n))
    A = np.asfortranarray(B + B.T)
    X = synth.gaussian_block(n, p, seed=3)
    Y = lb.spmm_dense(torch.from_numpy(A).cuda(), dev(torch, X)).cpu().numpy()
    ref = oracle.apply(A, X)
    scale = np.abs(A) @ np.abs(X)
    assert np.all(np.abs(Y - ref) <= 4 * np.finfo(float).eps * n * scale)


@pytest.mark.parametrize("n,p,q", [(1, 1, 1), (33, 5, 3), (10007, 16, 16), (100003, 48, 48), (4099, 96, 40), (777, 96, 96)])
def test_gram_matches_oracle(n, p, q):
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    X = synth.gaussian_block(n, p, seed=5)
    Y = synth.gaussian_block(n, q, seed=6)
    Cg = lb.gram(dev(torch, X), dev(torch, Y)).cpu().numpy()
    ref = oracle.gram(X, Y)
    scale = np.abs(X).T @ np.abs(Y)
    assert np.all(np.abs(Cg - ref) <= 8 * np.finfo(float).eps * np.log2(n + 2) * 16 * scale + 1e-300)


@pytest.mark.parametrize("two_stage", [False, True])
@pytest.mark.parametrize("s", [1, 2, 5, 12, 48, 95, 96])
def test_syev_matches_oracle_jacobi(s, two_stage):
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    g = np.random.default_rng(s)
    a = g.standard_normal((s, s))
    a = 0.5 * (a + a.T)
    lam, U = lb.syev(torch.from_numpy(a).cuda(), two_stage=two_stage)
    lam, U = lam.cpu().numpy(), U.cpu().numpy()
    lr, Ur, _ = oracle.jacobi_eig(a)
    nrm = max(1.0, np.linalg.norm(a))
    assert np.max(np.abs(lam - lr)) <= 1e-13 * nrm
    assert np.max(np.abs(U.T @ U - np.eye(s))) <= 1e-13 * s
    for j in range(s):  # simple eigenvalues: vectors agree up to sign
        assert abs(abs(U[:, j] @ Ur[:, j]) - 1) <= 1e-10


def test_ortho_matches_oracle_cholqr():
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    g = np.random.default_rng(7)
    X = g.standard_normal((30011, 12)) @ np.diag(10.0 ** np.linspace(0, 6, 12))
    Q, st = lb.ortho(dev(torch, X))
    Q = Q.cpu().numpy()
    Qr, str_ = oracle.ortho(np.asfortranarray(X))
    assert np.max(np.abs(Q.T @ Q - np.eye(12))) <= 1e-14
    assert np.max(np.abs(Q - Qr)) <= 1e-11
    assert st["passes"] == str_["passes"]


def test_ortho_shifted_path():
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    g = np.random.default_rng(3)
    U, _ = np.linalg.qr(g.standard_normal((3000, 8)))
    Vt, _ = np.linalg.qr(g.standard_normal((8, 8)))
    X = U @ np.diag(np.logspace(0, -12, 8)) @ Vt
    Q, st = lb.ortho(dev(torch, X))
    Q = Q.cpu().numpy()
    assert st["shifts"] >= 1 and st["passes"] <= 4
    assert np.max(np.abs(Q.T @ Q - np.eye(8))) <= 1e-14
    assert max_subspace_angle(Q, U) < 1e-3


def test_ortho_against_matches_properties_and_oracle():
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    g = np.random.default_rng(5)
    Y, _ = np.linalg.qr(g.standard_normal((40000, 20)))
    Xt = Y @ g.standard_normal((20, 6)) + 1e-9 * g.standard_normal((40000, 6))
    Q, st = lb.ortho_against(dev(torch, Xt), dev(torch, Y))
    Q = Q.cpu().numpy()
    Qr, str_ = oracle.ortho_against(np.asfortranarray(Xt), np.asfortranarray(Y))
    assert np.max(np.abs(Y.T @ Q)) <= 1e-14
    assert np.max(np.abs(Q.T @ Q - np.eye(6))) <= 1e-14
    assert max_subspace_angle(Q, Qr) <= 1e-6
    assert st["passes"] >= 2


def _f32_block(torch, X, ld):
    """float32 row-major copy of X with leading dimension ld (a multiple of 4)."""
    n, p = X.shape
    buf = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    buf[:, :p] = torch.from_numpy(X.astype(np.float32)).cuda()
    return buf[:, :p]


@pytest.mark.parametrize("n,p,band", [(50_001, 21, -1), (50_001, 16, 16), (20_011, 7, 0), (4_099, 32, 64),
                                      (3_001, 5, -2), (1, 1, -1), (2_000, 3, 2048), (30_011, 12, 256)])
def test_spmm_csr_f32_split_matches_oracle(n, p, band):
    """FP32 band / long-range split product against the FP64 oracle on the FP32-rounded
    operands: |Y - A32 X32| <= (nnz_row + 2) eps32 (|A32| |X32|) entrywise."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    a = synth.sparse_ci(n=n, seed=n) if n >= 600 else synth.tridiag_toeplitz(max(n, 1), 2.0, -1.0)
    X = synth.gaussian_block(a.n, p, seed=7)
    t = lb.upload_csr(a)
    ld = (p + 3) // 4 * 4
    Y, used = lb.spmm_csr_f32(t["row_ptr"], t["col_idx"], t["val"], _f32_block(torch, X, ld), band=band)
    Y = Y.cpu().numpy().astype(np.float64)
    a32 = synth.CSR(a.n, a.row_ptr, a.col_idx, a.val.astype(np.float32).astype(np.float64), a.diag)
    X32 = X.astype(np.float32).astype(np.float64)
    ref = oracle.apply(a32, X32)
    scale = np.abs(a32.to_scipy()) @ np.abs(X32)
    nz = int(np.max(np.diff(a.row_ptr))) + 2
    assert np.all(np.abs(Y - ref) <= nz * np.finfo(np.float32).eps * scale + 1e-30)
    if band >= 0:
        assert used == band
    elif band == -2:
        assert used == -1


@pytest.mark.parametrize("two_stage", [False, True])
@pytest.mark.parametrize("s", [7, 63, 96])
def test_syev_clustered_and_repeated_eigenvalues(s, two_stage):
    """Repeated and 1e-12-close eigenvalues: eigenvalues to 1e-13 ||a||, U orthonormal to
    1e-13 s and a U = U diag(lam) to 1e-13 ||a|| (vectors of a cluster are not unique)."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    g = np.random.default_rng(1000 + s)
    lam = np.sort(g.uniform(-1.0, 1.0, s))
    lam[: s // 3] = lam[0]                       # a repeated eigenvalue
    lam[s // 3: s // 3 + 3] = lam[s // 3] + np.array([0.0, 1e-12, 2e-12])  # a tight cluster
    lam = np.sort(lam)
    Q, _ = np.linalg.qr(g.standard_normal((s, s)))
    a = (Q * lam) @ Q.T
    a = 0.5 * (a + a.T)
    lg, U = lb.syev(torch.from_numpy(a).cuda(), two_stage=two_stage)
    lg, U = lg.cpu().numpy(), U.cpu().numpy()
    nrm = max(1.0, np.linalg.norm(a))
    assert np.max(np.abs(lg - lam)) <= 1e-13 * nrm
    assert np.max(np.abs(U.T @ U - np.eye(s))) <= 1e-13 * s
    assert np.max(np.abs(a @ U - U * lg)) <= 1e-13 * nrm


@pytest.mark.parametrize("s", [3, 21, 63, 96])
def test_syev_two_stage_fp32_polish(s):
    """Two-stage solve stopped at 1e-10 (FP32 rotations in its last stage), as the FP32
    phase of the mixed form runs it, on a graded spectrum with a cluster: eigenvalues and
    residuals to 1e-9 ||a||, U orthonormal to 1e-9."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    g = np.random.default_rng(2000 + s)
    lam = np.sort(np.concatenate([g.uniform(0.0, 0.05, s // 3), g.uniform(0.05, 20.0, s - s // 3)]))
    if s > 6:
        lam[2:5] = lam[2] + np.array([0.0, 1e-9, 3e-9])
    lam = np.sort(lam)
    Q, _ = np.linalg.qr(g.standard_normal((s, s)))
    a = (Q * lam) @ Q.T
    a = 0.5 * (a + a.T)
    lg, U = lb.syev(torch.from_numpy(a).cuda(), two_stage=True, tol=1e-10)
    lg, U = lg.cpu().numpy(), U.cpu().numpy()
    nrm = max(1.0, np.linalg.norm(a))
    assert np.max(np.abs(lg - lam)) <= 1e-9 * nrm
    assert np.max(np.abs(U.T @ U - np.eye(s))) <= 1e-9
    assert np.max(np.abs(a @ U - U * lg)) <= 1e-9 * nrm


def test_spmm_csr_f32_split_empty_rows_and_heavy_rows():
    """Split FP32 product on a CI-like matrix where every 7th row (and column) is empty, a
    few rows carry many long-range entries and a block of rows carries a dense band (its
    64-row sub-blocks exceed the shared-memory staging cap and are read from global
    memory): empty rows give zero rows of Y, long rows are summed in full."""
    torch = cuda()
    import scipy.sparse as sp
    import paper_2305_06668_gb300 as lb
    a = synth.sparse_ci(n=30_011, seed=77)
    m = a.to_scipy().tolil()
    keep = np.ones(a.n, dtype=bool)
    keep[::7] = False
    g = np.random.default_rng(5)
    heavy = g.choice(np.flatnonzero(keep), 5, replace=False)
    for r in heavy:  # 150 long-range partners each, mirrored
        cols = g.choice(np.flatnonzero(keep), 150, replace=False)
        v = g.normal(0, 0.005, 150)
        for c, x in zip(cols, v):
            if c != r:
                m[r, c] = x
                m[c, r] = x
    for r in range(8001, 8129):  # a dense band block: sub-blocks larger than the staging cap
        cols = r + g.choice(np.arange(-200, 201), 60, replace=False)
        for c in cols:
            if c != r:
                x = g.normal(0, 0.005)
                m[r, c] = x
                m[c, r] = x
    m = m.tocsr()
    D = sp.diags(keep.astype(float))
    m = (D @ m @ D).tocsr()
    m.sort_indices()
    m.eliminate_zeros()
    b = synth.CSR(a.n, m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data.astype(np.float64),
                  m.diagonal().astype(np.float64))
    assert np.count_nonzero(np.diff(b.row_ptr) == 0) >= a.n // 7
    p = 21
    X = synth.gaussian_block(b.n, p, seed=8)
    t = lb.upload_csr(b)
    Y, used = lb.spmm_csr_f32(t["row_ptr"], t["col_idx"], t["val"], _f32_block(torch, X, 24), band=-1)
    Y = Y.cpu().numpy().astype(np.float64)
    b32 = synth.CSR(b.n, b.row_ptr, b.col_idx, b.val.astype(np.float32).astype(np.float64), b.diag)
    X32 = X.astype(np.float32).astype(np.float64)
    ref = oracle.apply(b32, X32)
    scale = np.abs(b32.to_scipy()) @ np.abs(X32)
    nz = int(np.max(np.diff(b.row_ptr))) + 2
    assert used >= 0
    assert np.all(Y[~keep] == 0.0)
    assert np.all(np.abs(Y - ref) <= nz * np.finfo(np.float32).eps * scale + 1e-30)


@pytest.mark.parametrize("n,p,q,ld", [(1, 1, 1, 4), (97, 5, 3, 8), (10_007, 21, 21, 24), (100_003, 63, 63, 64),
                                      (50_001, 42, 21, 44), (4_099, 96, 40, 96), (7_001, 96, 96, 96),
                                      (20_011, 16, 16, 17)])
def test_gram_f32_matches_oracle(n, p, q, ld):
    """FP32 Gram (tensor-core 3xTF32 path when ld is a multiple of 4, FP32 FMA otherwise)
    against the FP64 oracle on the FP32-rounded blocks: |C - ref| <= 2^-19 |X|^T |Y| + a
    term for the FP32 sums over the rows of one CTA."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    X = synth.gaussian_block(n, p, seed=11).astype(np.float32).astype(np.float64)
    Y = synth.gaussian_block(n, q, seed=12).astype(np.float32).astype(np.float64)
    def dev32(M):
        buf = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
        buf[:, :M.shape[1]] = torch.from_numpy(M.astype(np.float32)).cuda()
        return buf[:, :M.shape[1]]
    Cg = lb.gram_f32(dev32(X), dev32(Y)).cpu().numpy()
    ref = oracle.gram(X, Y)
    scale = np.abs(X).T @ np.abs(Y)
    rows_per_cta = max(64, n // 304 + 64)
    tol = (2.0 ** -19 + rows_per_cta * np.finfo(np.float32).eps) * scale + 1e-30
    assert np.all(np.abs(Cg - ref) <= tol)


@pytest.mark.parametrize("n,ws,ld,q,mode", [
    (7001, (21, 21, 21), 24, 21, "pair_norm"),      # X, AX = [X W P] u_x with residual norms
    (200_000, (21, 21, 21), 24, 21, "pair_norm"),   # several 256-row chunks per CTA, ragged end
    (100_003, (21, 17, 9), 24, 19, "pair"),         # P, AP = V u_p
    (50_001, (21, 14), 24, 14, "base_inplace"),     # W -= Y C (alpha = -1, W is base and output)
    (30_011, (21,), 24, 16, "right_inplace"),       # W <- W S, q < w
    (20_000, (32, 32, 32), 32, 32, "pair_norm"),    # s = 96, q = 32
    (4_099, (3, 4), 8, 5, "plain"),
    (1, (2,), 4, 2, "pair_norm"),
    (9_001, (21, 5), 21, 13, "plain"),              # row stride not a multiple of 4: general kernel
])
def test_update_f32_matches_oracle(n, ws, ld, q, mode):
    """FP32 block update X = base + alpha [V_g] U (and AX, residual norms) against the
    oracle's FP64 product of the same FP32-rounded V and U: |X - ref| <= (s + 2) 2^-24 |V| |U|
    per element (FP32 FMA chain over s terms, then the scale and the base add)."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    s = sum(ws)
    r32 = lambda M: M.astype(np.float32).astype(np.float64)
    Vs = [r32(synth.gaussian_block(n, w, seed=100 + i)) for i, w in enumerate(ws)]
    AVs = [r32(synth.gaussian_block(n, w, seed=200 + i)) for i, w in enumerate(ws)]
    U = synth.gaussian_block(s, q, seed=7) / np.sqrt(s)
    lam = np.linspace(-1.0, 2.0, q)
    alpha = -1.0 if mode == "base_inplace" else 1.0

    def block32(M, stride):
        buf = torch.full((n, stride), float("nan"), dtype=torch.float32, device="cuda")  # padding poisoned
        buf[:, :M.shape[1]] = torch.from_numpy(M.astype(np.float32)).cuda()
        return buf[:, :M.shape[1]]

    Vd = [block32(M, ld) for M in Vs]
    AVd = [block32(M, ld) for M in AVs]
    Ud = torch.from_numpy(U).cuda()
    Vcat, AVcat = np.hstack(Vs), np.hstack(AVs)
    U32 = r32(U)
    ref = oracle.gram(Vcat.T.copy(), U32)          # (n x s)(s x q) as a Gram over the s rows
    scale = np.abs(Vcat) @ np.abs(U32)
    tol = (s + 2) * 2.0 ** -24 * scale + 1e-30
    if mode in ("pair_norm", "pair"):
        X, AX, *rest = lb.update_f32(Vd, Ud, AV=AVd, lam=torch.from_numpy(lam).cuda(),
                                     resnorm=(mode == "pair_norm"))
        aref = oracle.gram(AVcat.T.copy(), U32)
        atol = (s + 2) * 2.0 ** -24 * (np.abs(AVcat) @ np.abs(U32)) + 1e-30
        Xh, AXh = X.cpu().numpy().astype(np.float64), AX.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(Xh - ref) <= tol)
        assert np.all(np.abs(AXh - aref) <= atol)
        if rest:
            # the residual of the FP32 results, formed in FP32 per element and summed in FP64
            R = AXh - Xh * lam[None, :]
            rn_ref = np.sqrt(np.sum(R * R, axis=0))
            rtol = 8 * 2.0 ** -24 * np.sqrt(np.sum((np.abs(AXh) + np.abs(Xh * lam[None, :])) ** 2, axis=0))
            assert np.all(np.abs(rest[0] - rn_ref) <= rtol + 1e-300)
    elif mode == "base_inplace":
        W0 = r32(synth.gaussian_block(n, q, seed=9))
        W = block32(W0, ld)
        out = lb.update_f32(Vd, Ud, alpha=alpha, base=W, X=W)
        assert out.data_ptr() == W.data_ptr()
        Wh = W.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(Wh - (W0 - ref)) <= tol + 2.0 ** -24 * np.abs(W0))
    elif mode == "right_inplace":
        out = lb.update_f32(Vd, Ud, X=Vd[0][:, :q])
        Wh = Vd[0][:, :q].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(Wh - ref) <= tol)
        # the columns past q are left as they were
        assert np.array_equal(Vd[0][:, q:].cpu().numpy(), Vs[0][:, q:].astype(np.float32))
    else:
        X = lb.update_f32(Vd, Ud)
        assert np.all(np.abs(X.cpu().numpy().astype(np.float64) - ref) <= tol)


def test_update_f32_staged_and_general_layouts_agree():
    """The staged kernel (16-byte rows, ld a multiple of 4) and the general-layout kernel
    (here ld = 23) run the same FMA chain per element and form the residual AX - lam X
    with one fused multiply-add, so X and AX agree bit for bit and the residual norms
    differ only by the order of the per-row partial sums."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    n, ws, q = 70_001, [21, 21, 21], 21
    s = sum(ws)
    Vs = [synth.gaussian_block(n, w, seed=300 + i).astype(np.float32) for i, w in enumerate(ws)]
    AVs = [synth.gaussian_block(n, w, seed=400 + i).astype(np.float32) for i, w in enumerate(ws)]
    U = torch.from_numpy(synth.gaussian_block(s, q, seed=8) / np.sqrt(s)).cuda()
    lam = torch.from_numpy(np.linspace(-1.0, 2.0, q)).cuda()
    out = {}
    for ld in (24, 23):
        def block32(M):
            buf = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
            buf[:, :M.shape[1]] = torch.from_numpy(M).cuda()
            return buf[:, :M.shape[1]]
        zero = np.zeros((n, q), dtype=np.float32)
        X, AX, rn = lb.update_f32([block32(M) for M in Vs], U, AV=[block32(M) for M in AVs], lam=lam,
                                  X=block32(zero), AX=block32(zero), resnorm=True)
        out[ld] = (X.cpu().numpy(), AX.cpu().numpy(), np.asarray(rn))
    assert np.array_equal(out[24][0], out[23][0]) and np.array_equal(out[24][1], out[23][1])
    assert np.all(np.abs(out[24][2] - out[23][2]) <= 1e-6 * out[24][2])


def test_fma_rate_probe_is_plausible():
    """The FMA-rate probe (the denominator of the FMA-bound rooflines) returns rates inside
    what the part can do: FP64 near 2 FMA per clock per SM, FP32 near 128."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    f64 = lb.probe_fma_rate(fp64=True)
    f32 = lb.probe_fma_rate(fp64=False)
    ghz_max = 2.2  # above the part's 2.07 GHz boost clock
    assert 0.0 < f64 <= sms * 4 * ghz_max * 1e-3 * 1.05
    assert f64 * 8 < f32 <= sms * 256 * ghz_max * 1e-3 * 1.05
