"""Pins of the FP64 policy-network oracle: finite differences, closed forms,
Adam's published special cases (Kingma and Ba, ICLR 2015, Algorithm 1), the
action rule on hand-built networks, and an Adam fit to a target the network
can represent.  CPU only."""
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


# ---- Adam (Kingma and Ba 2015, Algorithm 1: beta1 = 0.9, beta2 = 0.999, eps = 1e-8) -----

def _trained_mask():
    keep = np.ones(mlp.N_PARAMS, bool)
    keep[:2 * mlp.N_IN] = False  # input mean and scale are not trained
    return keep


def test_adam_first_step_is_lr_times_sign():
    """From zero moments the bias-corrected moments at t = 1 are exactly g and
    g^2, so every weight moves by lr * g / (|g| + eps): about lr against the
    sign of its gradient, whatever the gradient's size."""
    rng = np.random.default_rng(11)
    p = random_params(rng)
    g = rng.normal(0, 1, mlp.N_PARAMS) * 10.0 ** rng.integers(-3, 4, mlp.N_PARAMS)
    z = np.zeros(mlp.N_PARAMS)
    lr = 0.01
    p1, m1, v1 = mlp.adam_step(p, g, z, z, 1, lr=lr)
    k = _trained_mask()
    assert np.allclose(p1[k], p[k] - lr * g[k] / (np.abs(g[k]) + 1e-8), rtol=0, atol=1e-14)
    assert np.all(np.abs(np.abs(p1[k] - p[k]) - lr) < 1e-6 * lr + lr * 1e-8 / np.abs(g[k]))
    assert np.array_equal(p1[~k], p[~k])
    # the first moment takes (1 - beta1) of the gradient, the second (1 - beta2) of its square
    assert np.allclose(m1, 0.1 * g, rtol=1e-15, atol=0)
    assert np.allclose(v1, 0.001 * g * g, rtol=1e-12, atol=0)


def test_adam_constant_gradient_keeps_unit_steps():
    """Under a constant gradient the bias-corrected moments stay g and g^2 at
    every t (m_t = (1 - beta1^t) g, v_t = (1 - beta2^t) g^2), so after t steps
    each weight has moved t * lr * g / (|g| + eps).  Without the bias
    correction the first steps would be about 3x too large (0.1 / sqrt(0.001))."""
    rng = np.random.default_rng(12)
    p0 = random_params(rng)
    g = rng.normal(0, 2, mlp.N_PARAMS)
    m = np.zeros(mlp.N_PARAMS)
    v = np.zeros(mlp.N_PARAMS)
    p = p0.copy()
    lr = 1e-3
    k = _trained_mask()
    for t in range(1, 11):
        p, m, v = mlp.adam_step(p, g, m, v, t, lr=lr)
        want = p0[k] - t * lr * g[k] / (np.abs(g[k]) + 1e-8)
        assert np.allclose(p[k], want, rtol=0, atol=1e-12), t


def test_adam_two_steps_worked_by_hand():
    """Gradient +1 then -3 on every weight, lr = 1:
    m_2 = 0.9 * 0.1 * 1 + 0.1 * (-3) = -0.21,
    v_2 = 0.999 * 0.001 * 1 + 0.001 * 9 = 0.009999,
    m_hat = -0.21 / (1 - 0.9^2) = -21/19, v_hat = 0.009999 / (1 - 0.999^2) = 9999/1999,
    second step = m_hat / (sqrt(v_hat) + eps) = -0.494189831087445 (worked out by
    hand from those fractions).  Swapping beta1 and beta2, or applying either to
    the wrong moment, gives another value."""
    p = np.zeros(mlp.N_PARAMS)
    z = np.zeros(mlp.N_PARAMS)
    p1, m1, v1 = mlp.adam_step(p, np.ones(mlp.N_PARAMS), z, z, 1, lr=1.0)
    p2, m2, v2 = mlp.adam_step(p1, np.full(mlp.N_PARAMS, -3.0), m1, v1, 2, lr=1.0)
    k = _trained_mask()
    assert np.allclose(m2, -0.21, rtol=1e-14, atol=0)
    assert np.allclose(v2, 0.009999, rtol=1e-12, atol=0)
    step2 = p1[k] - p2[k]
    assert np.allclose(step2, -0.494189831087445, rtol=1e-12, atol=0)
    assert np.allclose(p1[k], -1.0 / (1.0 + 1e-8), rtol=1e-15)


def test_adam_epsilon_is_outside_the_square_root():
    """For a gradient far below eps the first step is lr * g / (g + eps), about
    lr * g / eps; with eps under the square root it would be lr * g / sqrt(eps)."""
    g = np.full(mlp.N_PARAMS, 1e-12)
    z = np.zeros(mlp.N_PARAMS)
    p1, _, _ = mlp.adam_step(np.zeros(mlp.N_PARAMS), g, z, z, 1, lr=1.0)
    k = _trained_mask()
    assert np.allclose(-p1[k], 1e-12 / (1e-12 + 1e-8), rtol=1e-12, atol=0)


# ---- the action rule ------------------------------------------------------------------

def _constant_outputs(values):
    """A network whose outputs are `values` for every input (W3 = 0, b3 = values)."""
    p = random_params(np.random.default_rng(13))
    P = mlp.unpack(p)
    P["W3"][:] = 0
    P["b3"][:] = values
    return p


def test_predict_action_takes_the_smallest_allowed_output():
    X = np.zeros((3, mlp.N_IN))
    p = _constant_outputs([3.0, 1.0, 2.0, 0.5, 9.0, 9.0, 9.0, 9.0])
    assert mlp.predict_action(p, X, (0, 1, 2)).tolist() == [1, 1, 1]
    assert mlp.predict_action(p, X, (0, 2)).tolist() == [2, 2, 2]   # masked: 1 not allowed
    assert mlp.predict_action(p, X, (0,)).tolist() == [0, 0, 0]
    assert mlp.predict_action(p, X, (0, 1, 2, 3)).tolist() == [3, 3, 3]


def test_predict_action_ties_go_to_the_first_allowed():
    X = np.zeros((2, mlp.N_IN))
    p = _constant_outputs([1.0, 0.5, 0.5, 0.5, 7.0, 7.0, 7.0, 7.0])
    assert mlp.predict_action(p, X, (0, 1, 2)).tolist() == [1, 1]
    assert mlp.predict_action(p, X, (0, 2, 3)).tolist() == [2, 2]


def test_predict_action_follows_the_inputs():
    """Outputs 0..2 wired to inputs 0..2 through both ReLU layers (unit
    weights, a bias of 100 keeps every unit on): the action is the index of
    the smallest of the first three features, row by row."""
    p = np.zeros(mlp.N_PARAMS)
    P = mlp.unpack(p)
    P["sd"][:] = 1.0
    for k in range(3):
        P["W1"][k, k] = 1.0
        P["W2"][k, k] = 1.0
        P["W3"][k, k] = 1.0
    P["b1"][:3] = 100.0
    P["b3"][:3] = -100.0
    X = np.array([[3.0, -1.0, 2.0, 0, 0, 0], [0.5, 0.7, 0.6, 0, 0, 0], [-4.0, 5.0, -5.0, 0, 0, 0]])
    out, _ = mlp.forward(p, X)
    assert np.allclose(out[:, :3], X[:, :3])
    assert mlp.predict_action(p, X, (0, 1, 2)).tolist() == [1, 0, 2]
    assert mlp.predict_action(p, X, (0, 1)).tolist() == [1, 0, 0]
