"""Pins of the FP64 policy-network oracle: finite differences, closed forms,
and an Adam fit to a target the network can represent.  CPU only."""
import numpy as np

from oracle import mlp


def random_params(rng, scale=0.4):
    p = rng.normal(0, scale, mlp.N_PARAMS)
    P = mlp.unpack(p)
    P["mu"][:] = rng.normal(0, 1, mlp.N_IN)
    P["sd"][:] = rng.uniform(0.5, 2, mlp.N_IN)
    return p


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = random_params(rng)
    X = rng.normal(0, 2, (40, mlp.N_IN))
    a = rng.integers(0, 3, 40)
    y = rng.normal(0, 1, 40)
    L, g = mlp.loss_grad(p, X, a, y)
    assert abs(L - mlp.loss(p, X, a, y)) < 1e-12
    h = 1e-6
    for k in rng.choice(np.arange(2 * mlp.N_IN, mlp.N_PARAMS), 120, replace=False):
        e = np.zeros_like(p)
        e[k] = h
        fd = (mlp.loss(p + e, X, a, y) - mlp.loss(p - e, X, a, y)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd))
    assert np.all(g[:2 * mlp.N_IN] == 0)


def test_output_layer_closed_form():
    """With W3 = 0 the outputs are b3; the loss gradient on b3 is
    2/B * sum over rows taking action k of (b3[k] - y)."""
    rng = np.random.default_rng(1)
    p = random_params(rng)
    P = mlp.unpack(p)
    P["W3"][:] = 0
    X = rng.normal(0, 1, (25, mlp.N_IN))
    a = rng.integers(0, 3, 25)
    y = rng.normal(0, 1, 25)
    out, _ = mlp.forward(p, X)
    assert np.allclose(out, P["b3"])
    _, g = mlp.loss_grad(p, X, a, y)
    G = mlp.unpack(g)
    want = np.array([2.0 / 25 * np.sum(P["b3"][k] - y[a == k]) for k in range(mlp.N_OUT)])
    assert np.allclose(G["b3"], want)
    assert np.allclose(G["W2"], 0) and np.allclose(G["W1"], 0)


def test_dead_relu_passes_no_gradient():
    rng = np.random.default_rng(2)
    p = random_params(rng)
    P = mlp.unpack(p)
    P["b1"][:] = -1e6  # every first-layer unit off
    X = rng.normal(0, 1, (10, mlp.N_IN))
    _, g = mlp.loss_grad(p, X, rng.integers(0, 3, 10), rng.normal(0, 1, 10))
    G = mlp.unpack(g)
    assert np.all(G["W1"] == 0) and np.all(G["b1"] == 0) and np.all(G["W2"] == 0)


def test_features_definition():
    f = mlp.features([3], [10], [7], [5], 1000)
    assert np.allclose(f[0], [2.0, np.log2(11), 3.0, np.log2(6), np.log2(41) - np.log2(1001), np.log2(1 + 7 / 3)])


def test_adam_fits_a_representable_target():
    """A network whose action-0 output is a fixed function of the input is
    recovered by Adam on the masked loss (loss falls by 100x)."""
    rng = np.random.default_rng(3)
    teacher = random_params(rng, 0.6)
    X = rng.normal(0, 1.5, (400, mlp.N_IN))
    a = rng.integers(0, 3, 400)
    y = mlp.forward(teacher, X)[0][np.arange(400), a]
    p = random_params(np.random.default_rng(4), 0.3)
    mlp.unpack(p)["mu"][:] = mlp.unpack(teacher)["mu"]
    mlp.unpack(p)["sd"][:] = mlp.unpack(teacher)["sd"]
    L0 = mlp.loss(p, X, a, y)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in range(1, 3001):
        _, g = mlp.loss_grad(p, X, a, y)
        p, m, v = mlp.adam_step(p, g, m, v, t, lr=3e-3)
    assert mlp.loss(p, X, a, y) < L0 / 100
    assert np.all(p[:2 * mlp.N_IN] == teacher[:2 * mlp.N_IN])
