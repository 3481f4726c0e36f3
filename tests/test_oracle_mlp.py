"""Pins of the learned-scorer parts of the oracle: the FP64 network and its gradient
(finite differences), the C and NumPy forwards against each other, a hand-built network
whose function is known, the feature vector on a hand-worked example, and the learned rule
reducing to Algorithm 2's rule for weights that compute logit = 100 (n_e - n_z)/d - 50."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import gm
import oracle
from oracle import mlp


def _rand(seed, N=64):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(mlp.NPARAMS) * 0.3
    F = rng.standard_normal((N, 16))
    y = (rng.random(N) < 0.4).astype(float)
    return w, F, y


def test_gradient_matches_finite_differences():
    w, F, y = _rand(0)
    L, g = mlp.loss_and_grad(w, F, y)
    assert L == pytest.approx(mlp.loss(w, F, y), rel=1e-14)
    rng = np.random.default_rng(1)
    for p in rng.choice(mlp.NPARAMS, 60, replace=False).tolist() + [mlp.NPARAMS - 1, 0, 512, 1600]:
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[p] += h
        wm[p] -= h
        fd = (mlp.loss(wp, F, y) - mlp.loss(wm, F, y)) / (2 * h)
        assert abs(fd - g[p]) <= 1e-6 * max(1.0, abs(g[p])) + 1e-9, p


def test_c_and_numpy_forward_agree():
    w, F, _ = _rand(2, 200)
    o, _ = mlp.forward(w, F)
    np.testing.assert_allclose(oracle.mlp_logits(w, F), o, rtol=1e-12, atol=1e-12)


def test_a_hand_built_network_computes_its_function():
    # Layer 1 copies f0 and f1 through its ReLU, layer 2 forms relu(h0 - h1) and
    # relu(h1 - h0), the output adds them: logit = |relu(f0) - relu(f1)|.  A ReLU left
    # out or a weight matrix read transposed changes the value (without the second
    # layer's ReLU the two halves cancel); the other 14 features have zero weight.
    P = {name: np.zeros(size) for name, size in mlp.SIZES}
    W1 = P["W1"].reshape(mlp.NF, mlp.H)
    W2 = P["W2"].reshape(mlp.H, mlp.H)
    W1[0, 0] = W1[1, 1] = 1.0
    W2[0, 0] = W2[1, 1] = 1.0
    W2[1, 0] = W2[0, 1] = -1.0
    P["w3"][:2] = 1.0
    w = np.concatenate([P[name].ravel() for name, _ in mlp.SIZES])
    rng = np.random.default_rng(7)
    F = np.abs(rng.standard_normal((6, 16))) + 0.5
    F[:, :2] = [[0.7, 0.2], [0.2, 0.7], [-0.7, 0.2], [0.3, -0.9], [-0.5, -0.1], [1.25, 1.25]]
    want = np.abs(np.maximum(F[:, 0], 0.0) - np.maximum(F[:, 1], 0.0))
    np.testing.assert_allclose(oracle.mlp_logits(w, F), want, rtol=0, atol=1e-15)
    np.testing.assert_allclose(mlp.forward(w, F)[0], want, rtol=0, atol=1e-15)


def test_features_on_a_worked_example():
    # d = 5 rows, consensus value w = 1.0, sigma_n = 0.1
    rl = np.array([1.02, 0.97, 1.0, -0.3, 3.0])
    f = oracle.features(rl, 1.0, 2.8, 0.4, 0.05 + 1.3 + 2.0, 0.3 + 1.02 + 0.97 + 1.0 + 3.0, 0.1, 0.6, 0.7)
    # |r - w| / sigma: 0.2, 0.3, 0, 13 -> 8 (clip), 20 -> 8; sorted, padded with 8
    np.testing.assert_allclose(f[:7], [0.0, 0.2, 0.3, 8.0, 8.0, 8.0, 8.0], atol=1e-12)
    assert f[7] == pytest.approx(2.8 / 5) and f[8] == pytest.approx(0.4 / 5)
    assert f[9] == pytest.approx(math.log1p(10.0) / 5)
    assert f[10] == pytest.approx((6.29 - 3.35) / 6.29)
    assert (f[11], f[12]) == (0.6, 0.7)
    assert f[13] == pytest.approx((2.8 - 0.4) / 5)
    assert f[14] == 0 and f[15] == 0


def analytic_equivalent_bf16(d):
    """BF16 bits of weights with logit = 100 (n_e - n_z)/d - 50 (every value exact in BF16)."""
    w = np.zeros(mlp.NPARAMS, np.float32)
    P = dict()
    o = 0
    for name, size in mlp.SIZES:
        P[name] = o
        o += size
    w[P["W1"] + 13 * 32 + 0] = 100.0          # h1_0 = relu(100 f13)
    w[P["W2"] + 0 * 32 + 0] = 1.0             # h2_0 = relu(h1_0)
    w[P["w3"] + 0] = 1.0
    w[P["b3"]] = -50.0
    bits = (w.view(np.uint32) >> 16).astype(np.uint16)
    assert np.array_equal(oracle.bf16_to_f64(bits), w.astype(np.float64))
    return bits


def test_learned_rule_reduces_to_the_analytic_rule():
    # With d = 8 the analytic alpha is d/2 = 4 and logit >= 0 <=> (n_e - n_z)/8 >= 0.5.
    cfg = dict(n=3000, m=800, k=60, d=8, sigma_n=2e-3)
    I = gm.instance(seed=3, **cfg)
    A = sp.csr_matrix((np.ones(I.n * I.d), (I.rows.ravel(), np.repeat(np.arange(I.n), I.d))), shape=(I.m, I.n))
    y = (A @ I.x.astype(np.float64) + I.eta.astype(np.float64)).astype(np.float32).astype(np.float64)
    bits = analytic_equivalent_bf16(I.d)
    xa, sa, _ = oracle.decode(I.rows, y, I.k, sigma_n=I.sigma_n)
    xl, sl, _ = oracle.decode(I.rows, y, I.k, sigma_n=I.sigma_n, mlp_bf16=bits)
    np.testing.assert_allclose(xl, xa, rtol=1e-13, atol=1e-15)
    assert sl["rounds"] == sa["rounds"] and sl["accepted_rounds"] == sa["accepted_rounds"]
