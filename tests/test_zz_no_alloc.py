"""The allocation-free Gram entry point against the regular one (collected last).

lobpcg_gram_f64_noalloc serves callers that may not allocate device memory (for
example a serving loop whose GPU memory is sized once at start-up); it keeps its
partial sums in a fixed array inside the library.  Two calls in a row must each match
lobpcg_gram_f64 on its own inputs: the second, smaller call must not see anything the
first one left in the shared array.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import cuda, dev

pytestmark = pytest.mark.gpu


def _tol(X, Y, n):
    return 8 * np.finfo(float).eps * np.log2(n + 2) * 16 * (np.abs(X).T @ np.abs(Y)) + 1e-300


def test_noalloc_gram_matches_regular_entry_point_twice():
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    cases = [(200_003, 32, 32, 11), (5_001, 7, 20, 12)]  # second call smaller than the first
    for n, p, q, seed in cases:
        X = synth.gaussian_block(n, p, seed=seed)
        Y = synth.gaussian_block(n, q, seed=seed + 100)
        Xd, Yd = dev(torch, X), dev(torch, Y)
        ref = lb.gram(Xd, Yd).cpu().numpy()
        got = lb.gram_noalloc(Xd, Yd).cpu().numpy()
        tol = _tol(X, Y, n)
        assert np.all(np.abs(got - ref) <= 2 * tol)
        assert np.all(np.abs(got - X.T @ Y) <= tol)


def test_noalloc_gram_rejects_sizes_beyond_its_array():
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    X = dev(torch, synth.gaussian_block(100, 33, seed=1))
    Y = dev(torch, synth.gaussian_block(100, 32, seed=2))
    with pytest.raises(lb.LobpcgError) as e:
        lb.gram_noalloc(X, Y)
    assert e.value.status == lb.EINVAL and "1024" in str(e.value)
    # within p * q <= 1024 but wider than the Gram kernels take: also an argument error
    X1 = dev(torch, synth.gaussian_block(100, 1, seed=3))
    Y100 = dev(torch, synth.gaussian_block(100, 100, seed=4))
    with pytest.raises(lb.LobpcgError) as e:
        lb.gram_noalloc(X1, Y100)
    assert e.value.status == lb.EINVAL and "96" in str(e.value)
