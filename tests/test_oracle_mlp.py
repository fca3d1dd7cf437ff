"""Pins of the FP64 oracle of the learned preconditioner scale: closed forms for the
forward pass and central finite differences for both gradients."""
import numpy as np
import pytest

import oracle

H = 64
NP = H * 3 + H + H * H + H + H + 1


def params(seed, scale=0.3):
    g = np.random.default_rng(seed)
    return g.normal(0, scale, NP)


def test_param_count():
    assert oracle.mlp_num_params() == NP == 4481


def test_forward_special_cases():
    F = np.random.default_rng(0).normal(size=(7, 3))
    P = np.zeros(NP)
    assert np.allclose(oracle.mlp_forward(P, F), np.log(2.0), rtol=0, atol=1e-15)  # softplus(0)
    P[-1] = 2.5  # b3 only
    assert np.allclose(oracle.mlp_forward(P, F), np.log1p(np.exp(2.5)), rtol=0, atol=1e-15)
    # one active path: W1[0,0] = 1, W2[0,0] = 1, W3[0] = 1 -> z = relu(relu(f1))
    P = np.zeros(NP)
    P[0] = 1.0
    P[H * 3 + H] = 1.0
    P[H * 3 + H + H * H + H] = 1.0
    z = np.maximum(F[:, 0], 0.0)
    assert np.allclose(oracle.mlp_forward(P, F), np.log1p(np.exp(z)), rtol=1e-15, atol=1e-15)
    assert np.all(oracle.mlp_forward(params(3), F) > 0)


def test_backward_matches_central_differences():
    P = params(1)
    F = np.random.default_rng(2).normal(size=(5, 3))
    g = np.random.default_rng(3).normal(size=5)
    grad = oracle.mlp_backward(P, F, g)
    f = lambda p: float(g @ oracle.mlp_forward(p, F))
    idx = np.random.default_rng(4).choice(NP, 60, replace=False)
    idx = np.concatenate([idx, [0, 3 * H, 3 * H + H, NP - 66, NP - 1]])
    h = 1e-6
    for k in idx:
        e = np.zeros(NP)
        e[k] = h
        fd = (f(P + e) - f(P - e)) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, grad[k])


def test_loss_gradient_matches_central_differences_and_bounds():
    g = np.random.default_rng(5)
    N, ncol = 40, 3
    col = np.sort(g.integers(0, ncol, N)).astype(np.int32)
    q, e = g.normal(size=N), g.normal(size=N)
    s = np.exp(g.normal(size=N) * 0.3)
    far_we, far_ww = g.normal(size=ncol) * 0.1, np.abs(g.normal(size=ncol))
    ee = np.array([np.sum(e[col == c] ** 2) for c in range(ncol)]) + 0.5
    loss, d = oracle.mlp_loss(col, q, e, s, far_we, far_ww, ee)
    assert 0.0 <= loss <= 1.0
    h = 1e-7
    for i in range(N):
        sp, sm = s.copy(), s.copy()
        sp[i] += h
        sm[i] -= h
        fd = (oracle.mlp_loss(col, q, e, sp, far_we, far_ww, ee)[0] - oracle.mlp_loss(col, q, e, sm, far_we, far_ww, ee)[0]) / (2 * h)
        assert abs(fd - d[i]) <= 1e-6 * max(1.0, abs(fd))
    # a perfect direction (w parallel to e with no far part) has zero loss
    loss0, _ = oracle.mlp_loss(np.zeros(4, np.int32), np.ones(4), np.arange(1.0, 5.0), np.arange(1.0, 5.0),
                               [0.0], [0.0], [30.0])
    assert abs(loss0) < 1e-15
