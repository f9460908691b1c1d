"""Pins for the row-size predictor's CPU oracle: finite differences for the
gradient, hand-set weights for the forward pass, the closed form of Adam's
first step, and hand-computed row features. CPU only."""

import numpy as np

import oracle.mlp as mlp
import workloads as W


def test_param_count_and_layout():
    assert mlp.N_PARAMS == 6 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4673
    theta = np.arange(mlp.N_PARAMS, dtype=np.float64)
    p = mlp.unpack(theta)
    assert p["W1"][0, 1] == 1 and p["b1"][0] == 384 and p["W2"][0, 0] == 448
    assert p["b3"][0] == 4672
    assert np.array_equal(mlp.pack(p), theta)


def test_forward_hand_set_weights():
    theta = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(theta.copy())
    p["b3"][0] = 0.7
    X = np.random.default_rng(0).normal(size=(5, 6))
    y, _ = mlp.forward(mlp.pack(p), X)
    assert np.all(y == 0.7)
    # a single path x0 -> h1[0] -> h2[0] -> y computes relu(relu(x0)) * 2 - 1
    p["W1"][0, 0] = 1.0
    p["W2"][0, 0] = 1.0
    p["w3"][0] = 2.0
    p["b3"][0] = -1.0
    y, _ = mlp.forward(mlp.pack(p), X)
    assert np.allclose(y, np.maximum(X[:, 0], 0) * 2 - 1, rtol=0, atol=0)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = W.mlp_init(seed=3)
    theta[384:448] = rng.normal(0, 0.1, 64)   # nonzero biases
    X = rng.normal(size=(32, 6))
    t = rng.normal(size=32)
    L, g = mlp.backward(theta, X, t)
    assert abs(L - mlp.loss(mlp.forward(theta, X)[0], t)) < 1e-15 * max(1, L)
    h = 1e-6
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 200, replace=False),
                          [4672, 4671, 0, 383]])
    for j in idx:
        e = np.zeros_like(theta); e[j] = h
        num = (mlp.loss(mlp.forward(theta + e, X)[0], t)
               - mlp.loss(mlp.forward(theta - e, X)[0], t)) / (2 * h)
        assert abs(num - g[j]) <= 1e-6 * max(1.0, abs(num)), (j, num, g[j])


def test_adam_first_step_closed_form():
    # After one step m_hat = g and v_hat = g^2, so the update is
    # -lr * g / (|g| + eps).
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 1.0, 1.0, 1.0])
    th1, m, v = mlp.adam(th, g, np.zeros(4), np.zeros(4), step=1, lr=0.01)
    assert np.allclose(th1, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-15, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_decreases_loss_on_fixed_batch():
    rng = np.random.default_rng(2)
    X = rng.normal(size=(64, 6))
    t = X[:, 0] * 0.5 + 1.0
    theta = W.mlp_init(seed=0)
    m = np.zeros_like(theta); v = np.zeros_like(theta)
    losses = []
    for step in range(1, 201):
        L, g = mlp.backward(theta, X, t)
        losses.append(L)
        theta, m, v = mlp.adam(theta, g, m, v, step, lr=1e-2)
    assert losses[-1] < 0.05 * losses[0]


def test_features_hand_example():
    # A rows {0, 2}, {}, {1}; B row lengths 3, 1, 2.
    A = W.Csr(3, 3, np.array([0, 2, 2, 3], dtype=np.int32),
              np.array([0, 2, 1], dtype=np.int32), np.ones(3))
    B = W.Csr(3, 4, np.array([0, 3, 4, 6], dtype=np.int32),
              np.array([0, 1, 3, 2, 0, 3], dtype=np.int32), np.ones(6))
    X = mlp.features(A, B)
    want = np.log1p([[2, 5, 3, 2.5, 2], [0, 0, 0, 0, 0], [1, 1, 1, 1, 1]])
    assert np.allclose(X[:, :5], want, rtol=1e-15, atol=0)
    assert np.allclose(X[:, 5], np.log(np.array([1, 2, 3]) / 3), rtol=1e-15, atol=0)


def test_sizes():
    y = np.log1p(np.array([0.0, 9.5, 99.2]))
    assert mlp.sizes(y, 0.0).tolist() == [1, 10, 100]
    assert mlp.sizes(y, 0.1).tolist() == [1, 11, 110]
