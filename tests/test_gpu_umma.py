"""The FP32 Gram on the 5th-generation tensor cores (tcgen05.mma kind::tf32, TMA bulk copies,
TMEM accumulator) against the FP64 oracle on the FP32-rounded blocks.

Bound: |C - ref| <= (2^-19 + 24 eps_32 + chunks u_32) |X|^T |Y|: the 3xTF32 products keep
about 21 bits (2^-19 per product); the tensor core accumulates one chunk (32 or 64 rows, at
most 24 MMAs) in FP32, each MMA's addition off by at most one unit in the last place of a
partial sum bounded by the sum of |terms|; the chunks of one CTA are added with FP32
round-to-nearest adds (half a unit each); CTA sums are combined in FP64."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import cuda

pytestmark = pytest.mark.gpu


def _tol(n, scale):
    chunks = n // 152 // 32 + 2
    eps = float(np.finfo(np.float32).eps)
    return (2.0 ** -19 + 24 * eps + chunks * eps / 2) * scale + 1e-30


def _dev32(torch, M, ld):
    n, w = M.shape
    buf = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    buf[:, :w] = torch.from_numpy(M.astype(np.float32)).cuda()
    return buf[:, :w]


@pytest.mark.parametrize("n,p,q,ld", [(1, 1, 1, 4), (37, 3, 5, 8), (100_003, 21, 21, 24), (200_003, 63, 63, 64),
                                      (50_001, 64, 64, 64), (70_001, 42, 21, 44), (3_000, 17, 48, 48),
                                      (60_001, 96, 80, 96), (40_003, 70, 33, 72), (9_999, 33, 70, 72)])
def test_gram_tcgen05_matches_oracle(n, p, q, ld):
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    X = synth.gaussian_block(n, p, seed=n + 3).astype(np.float32).astype(np.float64)
    Y = synth.gaussian_block(n, q, seed=n + 4).astype(np.float32).astype(np.float64)
    Xd, Yd = _dev32(torch, X, ld), _dev32(torch, Y, ld)
    got = lb.gram_f32_tcgen05(Xd, Yd).cpu().numpy()
    ref = oracle.gram(X, Y)
    scale = np.abs(X).T @ np.abs(Y)
    tol = _tol(n, scale)
    err = np.abs(got - ref)
    assert np.all(err <= tol), float(np.max(err / (scale + 1e-300)))
    print("max err / scale", float(np.max(err / (scale + 1e-300))))
    # and it agrees with the warp-level mma.sync kernel to the same bound
    old = lb.gram_f32(Xd, Yd).cpu().numpy()
    assert np.all(np.abs(got - old) <= 2 * tol)


def test_gram_tcgen05_exact_on_small_integers():
    """Integers below 2^10: the hi parts are exact, the lo parts zero, every product and
    every FP32 sum up to 2^24 exact, so the result equals the integer Gram."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    g = np.random.default_rng(5)
    n, p = 8_192, 24
    X = g.integers(-16, 17, size=(n, p)).astype(np.float64)
    Y = g.integers(-16, 17, size=(n, p)).astype(np.float64)
    got = lb.gram_f32_tcgen05(_dev32(torch, X, 24), _dev32(torch, Y, 24)).cpu().numpy()
    assert np.array_equal(got, X.T @ Y)


def test_gram_tcgen05_same_block_and_offset_views():
    """X^T X (one block behind both operands: copied once, split once) and views that start
    16 bytes into their rows of a wider buffer (the last row's copy stops at the used
    columns)."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    n = 123_457
    for p, ld in [(21, 24), (63, 64), (96, 96)]:
        X = synth.gaussian_block(n, p, seed=p).astype(np.float32).astype(np.float64)
        Xd = _dev32(torch, X, ld)
        got = lb.gram_f32_tcgen05(Xd, Xd).cpu().numpy()
        scale = np.abs(X).T @ np.abs(X)
        assert np.all(np.abs(got - oracle.gram(X, X)) <= _tol(n, scale)), p
    F = synth.gaussian_block(n, 32, seed=9).astype(np.float32).astype(np.float64)
    buf = torch.from_numpy(np.ascontiguousarray(F, dtype=np.float32)).cuda()
    assert buf.stride(0) == 32
    Xv, Yv = buf[:, 4:25], buf[:, 8:31]
    got = lb.gram_f32_tcgen05(Xv, Yv).cpu().numpy()
    X, Y = F[:, 4:25], F[:, 8:31]
    assert np.all(np.abs(got - oracle.gram(X, Y)) <= _tol(n, np.abs(X).T @ np.abs(Y)))


def test_gram_tcgen05_rejects_unaligned_rows():
    """Rows that are not 16-byte aligned cannot be bulk-copied: an argument error (the
    solver then uses the warp-level kernel)."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    X = _dev32(torch, synth.gaussian_block(1000, 21, seed=1), 22)
    with pytest.raises(lb.LobpcgError) as e:
        lb.gram_f32_tcgen05(X, X)
    assert e.value.status == lb.EINVAL
