"""Pins for the triage oracle (numpy FP64): each checked against something
other than itself -- numpy's symmetric eigen-solver on a planted spectrum,
finite differences, closed forms and numpy's quantile function."""
import math

import numpy as np
import pytest

from oracle import triage_oracle as TO


def test_ritz_values_reach_a_planted_spectrum():
    rng = np.random.default_rng(0)
    N, d = 400, 64
    lam = np.concatenate([np.geomspace(50.0, 5.0, 16), np.full(d - 16, 0.2)])
    Q1, _ = np.linalg.qr(rng.standard_normal((N, d)))
    Q2, _ = np.linalg.qr(rng.standard_normal((d, d)))
    Z = Q1 @ np.diag(np.sqrt(lam * N)) @ Q2.T  # Z^T Z / N = Q2 diag(lam) Q2^T
    want = np.sort(np.linalg.eigvalsh(Z.T @ Z / N))[::-1][:16]
    got = TO.ritz_values(Z, iters=40)
    assert np.allclose(got, want, rtol=1e-8)
    assert np.allclose(want, lam[:16], rtol=1e-8)


def test_mgs_is_orthonormal_and_spans_the_input():
    rng = np.random.default_rng(1)
    W = rng.standard_normal((50, 16))
    V = TO.mgs(W)
    assert np.allclose(V.T @ V, np.eye(16), atol=1e-12)
    # same column space: projecting W onto span(V) leaves it unchanged
    assert np.allclose(V @ (V.T @ W), W, atol=1e-10)


def test_start_block_is_fixed_and_bounded():
    a, b = TO.start_block(40), TO.start_block(40)
    assert (a == b).all() and a.min() >= -0.5 and a.max() < 0.5
    assert np.abs(np.corrcoef(a.T)[np.triu_indices(16, 1)]).max() < 0.6


def _params(seed=3):
    rng = np.random.default_rng(seed)
    _, _, n = TO.param_layout()
    return (rng.standard_normal(n) * 0.1).astype(np.float32).astype(np.float64)


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = _params()
    F = rng.standard_normal((7, TO.N_FEAT))
    target = rng.standard_normal((7, TO.N_OUT))

    def loss_of(y):
        return TO.pinball(y, target)[0]

    y, cache = TO.mlp_forward(params, F)
    _, dy = TO.pinball(y, target)
    g = TO.mlp_backward(params, cache, dy)
    # finite differences with respect to the (BF16-rounded) weights: perturb the
    # rounded weights through the layer maths directly
    W1, b1, W2, b2, W3, b3 = TO.unpack(params)
    W1r, W2r, W3r = TO.bf16_round(W1), TO.bf16_round(W2), TO.bf16_round(W3)

    def fwd(W1r, b1, W2r, b2, W3r, b3):
        h1 = np.maximum(F @ W1r + b1, 0)
        h2 = np.maximum(h1 @ W2r + b2, 0)
        return h2 @ W3r + b3

    grads = TO.unpack(g)
    base = [W1r, b1, W2r, b2, W3r, b3]
    eps = 1e-6
    # (layer parameter index, element)
    for j, idx in [(0, (3, 17)), (2, (100, 7)), (4, (5, 2)), (3, (11,)), (5, (4,)), (1, (200,))]:
        plus = [x.copy() for x in base]
        minus = [x.copy() for x in base]
        plus[j][idx] += eps
        minus[j][idx] -= eps
        fd = (loss_of(fwd(*plus)) - loss_of(fwd(*minus))) / (2 * eps)
        assert abs(fd - grads[j][idx]) <= 1e-6 + 1e-4 * abs(fd)


def test_pinball_closed_form_and_gradient():
    pred = np.array([[1.0, 2.0, 3.0, 0, 0, 0, 0, 0, 0]])
    target = np.array([[2.0, 1.0, 3.0, 0, 0, 0, 0, 0, 0]])
    loss, d = TO.pinball(pred, target)
    # u = [1, -1, 0, 0...]: 0.5*1 + (0.8-1)*(-1) = 0.7, mean over 9
    assert abs(loss - 0.7 / 9) < 1e-15
    assert abs(d[0, 0] + 0.5 / 9) < 1e-15 and abs(d[0, 1] - 0.2 / 9) < 1e-15


def test_null_quantiles_are_the_inverted_cdf():
    rng = np.random.default_rng(5)
    T = rng.standard_normal(9999)
    got = TO.null_quantiles(T)
    want = np.quantile(np.abs(T), TO.LEVELS, method="inverted_cdf")
    assert np.array_equal(got, want)


def test_predicted_p_at_the_knots_and_monotone():
    q = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0, 8.0, 9.0])
    for k in range(9):
        assert abs(TO.predict_p(q, q[k]) - (1 - TO.LEVELS[k])) < 1e-12
    ts = np.linspace(0, 12, 200)
    ps = [TO.predict_p(q, t) for t in ts]
    assert all(a >= b for a, b in zip(ps, ps[1:]))
    assert ps[0] == 1.0 and min(ps) >= 1e-4 - 1e-15


def test_adam_first_step_is_lr_times_sign():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    new, m, v = TO.adam(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> step = lr * g / (|g| + eps)
    assert np.allclose(new, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_bf16_round_agrees_with_the_c_oracle_rounding():
    from oracle import oracle as O

    rng = np.random.default_rng(11)
    v = np.concatenate([rng.standard_normal(500) * 10.0 ** rng.integers(-30, 30, 500),
                        [0.0, -0.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20]])
    v32 = v.astype(np.float32).astype(np.float64)
    got = TO.bf16_round(v32)
    want = np.array([O.round_to_bf16(float(x)) for x in v32])
    assert np.array_equal(got, want)
    assert got[-3] == 1.0 and got[-2] == 1.0 + 2.0 ** -6 and got[-1] == 1.0 + 2.0 ** -7  # ties to even, above the tie


def test_mlp_forward_hand_computed_network():
    """A network whose output is known in closed form pins the flat parameter
    layout (written here from its documented definition, not through
    `unpack`: [W1 19x256 | b1 256 | W2 256x256 | b2 256 | W3 256x9 | b3 9],
    weights input-major and row-major), both ReLUs (negative pre-activations
    must be zeroed) and the BF16 rounding of the weights:
      hidden1: h_i = relu(F_i - 1) for i < 9, h_19 = 2.5, h_23 = relu(3 F_2), h_30 = relu(-4) = 0;
      hidden2: g_i = 2 h_i for i < 9, g_19 = 2 h_19, g_23 = h_23, g_30 = relu(h_30 - 3) = 0,
               g_31 = relu(-1) = 0;
      output:  y_k = BF16(1 + 2^-10) g_k + 0.5 g_19 + 7 g_30 + 7 g_31 + k with BF16(1 + 2^-10) = 1,
               plus g_23 for k = 8."""
    H1, NF, NO = 256, 19, 9
    oW1, ob1 = 0, NF * H1
    oW2, ob2 = ob1 + H1, ob1 + H1 + H1 * H1
    oW3, ob3 = ob2 + H1, ob2 + H1 + H1 * NO
    total = ob3 + NO
    assert total == TO.param_layout()[2] == 73225
    w = np.zeros(total)
    W1 = lambda i, j: oW1 + i * H1 + j  # noqa: E731
    W2 = lambda i, j: oW2 + i * H1 + j  # noqa: E731
    W3 = lambda i, k: oW3 + i * NO + k  # noqa: E731
    for i in range(9):
        w[W1(i, i)] = 1.0
        w[ob1 + i] = -1.0
        w[W2(i, i)] = 2.0
        w[W3(i, i)] = 1.0 + 2.0 ** -10  # rounds to 1.0 in BF16
        w[ob3 + i] = float(i)
    w[ob1 + 19] = 2.5
    w[W2(19, 19)] = 2.0
    for k in range(NO):
        w[W3(19, k)] = 0.5
        w[W3(30, k)] = 7.0
        w[W3(31, k)] = 7.0
    w[W1(2, 23)] = 3.0   # input 2 -> hidden 23 (a transposed layout would route it elsewhere)
    w[W2(23, 23)] = 1.0
    w[W3(23, 8)] = 1.0
    w[ob1 + 30] = -4.0
    w[W2(30, 30)] = 1.0
    w[ob2 + 30] = -3.0
    w[ob2 + 31] = -1.0
    rng = np.random.default_rng(4)
    F = rng.uniform(-2.0, 3.0, size=(6, NF))
    y, _ = TO.mlp_forward(w, F)
    want = 2.0 * np.maximum(F[:, :9] - 1.0, 0.0) + 0.5 * 2.0 * 2.5 + np.arange(9.0)
    want[:, 8] += np.maximum(3.0 * F[:, 2], 0.0)
    assert np.allclose(y, want, rtol=0, atol=1e-12)
