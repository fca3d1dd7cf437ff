"""GPU kernels of the learned preconditioner (BF16 weights/activations, FP32 sums)
against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import cuda

pytestmark = pytest.mark.gpu
NP = 4481


def _params(seed):
    g = np.random.default_rng(seed)
    P = g.normal(0, 0.25, NP)
    P[-1] = 0.5413  # softplus(b3) ~ 1
    return P


def _bf16(x):
    """Round float64 to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    a = (a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000
    return a.astype(np.uint32).view(np.float32).astype(np.float64)


def test_forward_matches_oracle_at_bf16_precision():
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    P = _params(1)
    F = np.random.default_rng(2).normal(size=(20000, 3))
    s = lb.mlp_forward(torch.from_numpy(F.astype(np.float32)).cuda(), torch.from_numpy(P.astype(np.float32)).cuda())
    s = s.cpu().numpy()
    ref = oracle.mlp_forward(P, F)
    # bf16 rounding of weights and activations: ~3 significant digits
    assert np.median(np.abs(s - ref) / ref) < 1e-2
    assert np.max(np.abs(s - ref) / ref) < 8e-2
    # with the weights and inputs already bf16 values the only differences are the two
    # rounded activation layers
    s2 = lb.mlp_forward(torch.from_numpy(_bf16(F).astype(np.float32)).cuda(),
                        torch.from_numpy(_bf16(P).astype(np.float32)).cuda()).cpu().numpy()
    ref2 = oracle.mlp_forward(_bf16(P), _bf16(F))
    assert np.median(np.abs(s2 - ref2) / ref2) < 5e-3


def test_fp32_mode_matches_oracle_tightly():
    """Without BF16 rounding the kernels must reproduce the FP64 definition to FP32 accuracy."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    P = _params(7)
    F = np.random.default_rng(8).normal(size=(4000, 3))
    g = np.random.default_rng(9).normal(size=4000)
    Ft, Pt = torch.from_numpy(F.astype(np.float32)).cuda(), torch.from_numpy(P.astype(np.float32)).cuda()
    P32, F32 = P.astype(np.float32).astype(np.float64), F.astype(np.float32).astype(np.float64)
    s = lb.mlp_forward(Ft, Pt, bf16=False).cpu().numpy()
    assert np.max(np.abs(s - oracle.mlp_forward(P32, F32)) / oracle.mlp_forward(P32, F32)) < 1e-5
    grad = torch.zeros(NP, dtype=torch.float32, device="cuda")
    lb.mlp_backward(Ft, Pt, torch.from_numpy(g.astype(np.float32)).cuda(), grad, bf16=False)
    ref = oracle.mlp_backward(P32, F32, g.astype(np.float32).astype(np.float64))
    assert np.linalg.norm(grad.cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)


def test_backward_matches_oracle_gradient():
    """BF16 mode: the rounded activations (unit roundoff 2^-8) move the summed gradients
    by a few per cent of their norm."""
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    P = _bf16(_params(3))
    F = _bf16(np.random.default_rng(4).normal(size=(3000, 3)))
    g = np.random.default_rng(5).normal(size=3000)
    grad = torch.zeros(NP, dtype=torch.float32, device="cuda")
    lb.mlp_backward(torch.from_numpy(F.astype(np.float32)).cuda(), torch.from_numpy(P.astype(np.float32)).cuda(),
                    torch.from_numpy(g.astype(np.float32)).cuda(), grad)
    ref = oracle.mlp_backward(P, F, g)
    gg = grad.cpu().numpy()
    rel = np.linalg.norm(gg - ref) / np.linalg.norm(ref)
    blocks = [(0, 192), (192, 256), (256, 4352), (4352, 4416), (4416, 4480), (4480, 4481)]
    per = [float(np.linalg.norm(gg[a:b] - ref[a:b]) / max(np.linalg.norm(ref[a:b]), 1e-30)) for a, b in blocks]
    assert rel < 5e-2, (rel, per)
    # per-block agreement (W1, b1, W2, b2, W3, b3)
    for (a, b), r in zip(blocks, per):
        assert r <= 8e-2, (a, b, per)


def test_loss_and_adam():
    torch = cuda()
    import paper_2305_06668_gb300 as lb
    g = np.random.default_rng(6)
    N, ncol = 5000, 4
    col = np.sort(g.integers(0, ncol, N)).astype(np.int32)
    q, e = g.normal(size=N), g.normal(size=N)
    s = np.exp(g.normal(size=N) * 0.3)
    far_we, far_ww = g.normal(size=ncol) * 0.1, np.abs(g.normal(size=ncol))
    ee = np.array([np.sum(e[col == c] ** 2) for c in range(ncol)]) + 0.5
    q32, e32, s32 = (v.astype(np.float32).astype(np.float64) for v in (q, e, s))
    ref_loss, ref_d = oracle.mlp_loss(col, q32, e32, s32, far_we, far_ww, ee)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).cuda()
    loss, d = lb.mlp_loss(t(col, np.int32), t(q, np.float32), t(e, np.float32), t(s, np.float32),
                          t(far_we, np.float64), t(far_ww, np.float64), t(ee, np.float64))
    assert abs(loss - ref_loss) < 1e-10
    assert np.max(np.abs(d.cpu().numpy() - ref_d)) <= 1e-5 * np.max(np.abs(ref_d))
    # Adam: one step from zero moments moves every parameter by -lr * sign(grad)
    P = torch.zeros(NP, dtype=torch.float32, device="cuda")
    grad = torch.linspace(-1, 1, NP, dtype=torch.float32, device="cuda") + 1e-3
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    lb.mlp_adam(P, grad, m, v, 1, lr=0.01)
    assert torch.allclose(P, -0.01 * torch.sign(torch.linspace(-1, 1, NP, device="cuda") + 1e-3), atol=1e-6)
    assert float(grad.abs().max()) == 0.0
