"""Batched solve: every problem's result equals its one-by-one solve bit for bit, and
matches the oracle's eigenvalues."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import cuda
from tests.util import rel_eig_err

pytestmark = pytest.mark.gpu


def _problems(torch):
    import paper_2305_06668_gb300 as lb
    g = np.random.default_rng(3)
    specs = [(int(n), int(k)) for n, k in zip(g.integers(3000, 30000, 12), g.integers(1, 9, 12))]
    probs = []
    for p, (n, k) in enumerate(specs):
        a = synth.sparse_cfg1(n=n, seed=500 + p)
        probs.append((a, k, synth.diag_guess(a.diag, k, seed=500 + p, noise=0.0)))
    return probs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_equals_one_by_one_and_oracle(precision):
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    prec = lb.MIXED if precision == "mixed" else lb.FP64
    probs = _problems(torch)
    t = [lb.upload_csr(a) for a, _, _ in probs]
    x0 = [torch.from_numpy(x).cuda() for _, _, x in probs]
    streams = [torch.cuda.Stream() for _ in probs]
    solvers = [lb.Solver(**ti, precision=prec, stream=st) for ti, st in zip(t, streams)]
    res_b = lb.solve_batched(solvers, [k for _, k, _ in probs], [1e-8] * len(probs), x0, nthreads=6)
    for s, (a, k, _), x, rb in zip(solvers, probs, x0, res_b):
        r1 = s.solve(k, 1e-8, X0=x)
        assert rb.status == r1.status == 0
        assert np.array_equal(rb.evals, r1.evals)
        assert np.array_equal(rb.resnorms, r1.resnorms)
        assert torch.equal(rb.evecs, r1.evecs)
    for (a, k, x), rb in list(zip(probs, res_b))[:4]:
        ref = oracle.lobpcg(a, a.diag, k, x, tol=1e-8)
        assert np.max(rel_eig_err(rb.evals, ref.evals)) <= 1e-10
    for s in solvers:
        s.close()


def test_gpu_generator_follows_the_recipe():
    torch = cuda()
    t = synth.sparse_cfg1_torch(5000, seed=9)
    rp, ci, val, d = (v.cpu().numpy() for v in (t["row_ptr"], t["col_idx"], t["val"], t["diag"]))
    import scipy.sparse as sp
    A = sp.csr_matrix((val, ci, rp), shape=(5000, 5000))
    assert abs(A - A.T).max() == 0.0
    assert np.array_equal(A.diagonal(), d) and np.all(np.diff(d) >= 0)
    assert np.all(np.abs(d - 0.01 * np.arange(5000)) <= 0.005 + 0.01)
    off = A - sp.diags(d)
    assert 30 <= off.nnz / 5000 <= 33  # 16 per row mirrored, minus duplicates
    assert abs(np.std(off.data) - 0.01) < 0.001
