"""Pins for the learned-form oracle (oracle/mlp.py), independent of its own
code: torch's bfloat16 conversion, central finite differences in float64,
closed forms of a zero network and of a first Adam step, scipy's log-sigmoid,
and a hand-built visit record.  No GPU needed."""
import numpy as np
import pytest
import scipy.special
import torch

from oracle import mlp


def _params(rng, scale=0.3):
    return rng.standard_normal(mlp.PARAMS) * scale


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-6, 6, 20000)).astype(np.float32)
    # exact ties: a BF16 value plus half an ULP of BF16, both parities
    base = torch.tensor(rng.standard_normal(200), dtype=torch.bfloat16).float().numpy()
    ties = (base.view(np.uint32) | np.uint32(0x8000)).view(np.float32)
    x = np.concatenate([x, ties, np.float32([0.0, -0.0, 1.0, 3.0e38])])
    want = torch.from_numpy(x).to(torch.bfloat16).double().numpy()
    assert np.array_equal(mlp.bf16_round(x), want)


def test_zero_network_closed_form():
    p = np.zeros(mlp.PARAMS)
    p[mlp.OFF_B3] = 0.7
    X = np.random.default_rng(1).standard_normal((5, 8))
    y = np.array([0, 1, 1, 0, 1], dtype=float)
    z = mlp.forward(p, X)
    assert np.allclose(z, 0.7)
    loss, g = mlp.loss_grad(p, X, y)
    # softplus(b) - y b, mean over samples; d/db3 = mean(sigmoid(b) - y)
    assert loss == pytest.approx(np.mean(np.log1p(np.exp(0.7)) - y * 0.7), rel=1e-14)
    assert g[mlp.OFF_B3] == pytest.approx(np.mean(1.0 / (1.0 + np.exp(-0.7)) - y), rel=1e-14)
    assert np.all(g[:mlp.OFF_B3] == 0.0)


def test_loss_matches_scipy_log_sigmoid():
    rng = np.random.default_rng(2)
    p = _params(rng)
    X = rng.standard_normal((40, 8))
    y = (rng.random(40) < 0.5).astype(float)
    z = mlp.forward(p, X)
    want = -np.mean(y * scipy.special.log_expit(z) + (1 - y) * scipy.special.log_expit(-z))
    assert mlp.loss_grad(p, X, y)[0] == pytest.approx(want, rel=1e-13)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = _params(rng)
    X = rng.standard_normal((16, 8))
    y = (rng.random(16) < 0.5).astype(float)
    _, g = mlp.loss_grad(p, X, y, round_weights=False)
    idx = np.concatenate([rng.choice(mlp.OFF_B1, 20, replace=False), np.arange(mlp.OFF_B1, mlp.OFF_B1 + 5),
                          rng.choice(np.arange(mlp.OFF_W2, mlp.OFF_B2), 30, replace=False),
                          np.arange(mlp.OFF_B2, mlp.OFF_B2 + 5), np.arange(mlp.OFF_W3, mlp.OFF_W3 + 10),
                          [mlp.OFF_B3]])
    h = 1e-6
    for q in idx:
        e = np.zeros(mlp.PARAMS)
        e[q] = h
        fd = (mlp.loss_grad(p + e, X, y, False)[0] - mlp.loss_grad(p - e, X, y, False)[0]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-7 + 1e-5 * abs(g[q]), (q, fd, g[q])


def test_first_adam_step_closed_form():
    g = np.array([0.3, -2.0, 1e-9, 0.0])
    p0 = np.ones(4)
    p, m, v = mlp.adam_step(p0, np.zeros(4), np.zeros(4), g, 1, lr=0.01, eps=1e-8)
    # first step: m_hat = g, v_hat = g^2, so the step is lr g / (|g| + eps)
    assert np.allclose(p, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_record_and_features_by_hand():
    b = 2
    A = np.array([[4.0, 0.0, 2.0, -1.0], [0.0, 9.0, 0.0, 3.0], [2.0, 0.0, 1.0, 0.0], [-1.0, 3.0, 0.0, 16.0]])
    sg = np.array([1, -1, 1, 1])
    r = mlp.record(A, sg, b)
    # scaled I x J block: |2|/sqrt(4*1)=1, |-1|/sqrt(4*16)=1/8, 0, |3|/sqrt(9*16)=1/4
    assert r[0] == 1.0
    assert r[1] == pytest.approx(np.sqrt(1 + 1 / 64 + 1 / 16))
    assert r[3] == 6.5 and r[4] == 8.5
    # signs: I = (+, -), J = (+, +): opposite pairs are (-, +) twice
    assert r[5] == 0.5
    r[2] = 3.0
    f = mlp.features(r, 1, 5, 2, b, 8, 3, 30, 2.0 ** -10)
    assert f == pytest.approx([10 / 64, np.log2(r[1]) / 64, 0.75, 0.1, 0.5, np.log2(6.5 / 8.5) / 64, 3 / 8, 1.0])
