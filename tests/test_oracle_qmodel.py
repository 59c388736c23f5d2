"""Pins of the FP64 oracle of the learned-q form (oracle/qmodel.py), each
against something other than the oracle itself: central finite differences
for the backpropagated gradient, hand-computed Adam updates, a forward pass
through hand-set weights, features of a hand-made buffer, the label rule on
hand-made ladder results."""
import math

import numpy as np
import pytest

from oracle import qmodel as Q


def test_parameter_count():
    assert Q.NPARAM == 16 * 64 + 64 + 64 * 64 + 64 + 64 + 1


@pytest.mark.parametrize("seed,batch", [(0, 1), (1, 7), (2, 32)])
def test_gradient_matches_central_differences(seed, batch):
    rng = np.random.default_rng(seed)
    theta = Q.init_params(seed) + 0.05 * rng.standard_normal(Q.NPARAM)
    X = rng.standard_normal((batch, Q.NF))
    X[:, 0] = 1.0
    t = rng.uniform(1, 13, batch)
    loss, g = Q.mlp_backward(theta, X, t)
    assert loss == pytest.approx(Q.mse_loss(Q.mlp_forward(theta, X)[0], t))
    # every parameter block, including ReLU units that are off for some rows
    idx = rng.choice(Q.NPARAM, 300, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (Q.mse_loss(Q.mlp_forward(tp, X)[0], t) - Q.mse_loss(Q.mlp_forward(tm, X)[0], t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_adam_two_steps_by_hand():
    # g1 = +1, g2 = -1, lr = 0.1: m1 = 0.1, v1 = 0.001 -> both corrected to 1;
    # m2 = -0.01, v2 = 0.001999 -> corrected -0.01/0.19 and 1
    th = np.array([0.5])
    m = np.zeros(1)
    v = np.zeros(1)
    th, m, v = Q.adam_step(th, np.array([1.0]), m, v, 1, 0.1)
    assert th[0] == pytest.approx(0.5 - 0.1 / (1 + 1e-8), abs=1e-15)
    th, m, v = Q.adam_step(th, np.array([-1.0]), m, v, 2, 0.1)
    assert m[0] == pytest.approx(-0.01)
    assert v[0] == pytest.approx(0.001999)
    assert th[0] == pytest.approx(0.5 - 0.1 / (1 + 1e-8) + 0.1 * (0.01 / 0.19) / (1 + 1e-8),
                                  abs=1e-12)


def test_forward_through_hand_set_weights():
    theta = np.zeros(Q.NPARAM)
    p = Q.unpack(theta)
    p["W1"][0, 0] = 2.0      # h1_0 = relu(2 x0 + b1_0)
    p["W1"][1, 1] = -1.0     # h1_1 = relu(-x1)
    p["W2"][0, 0] = 3.0      # h2_0 = relu(3 h1_0)
    p["W2"][1, 0] = 1.0      #      + h1_1
    p["w3"][0] = 0.5
    p["b3"][0] = 1.0
    X = np.zeros((3, Q.NF))
    X[:, 0] = 1.0
    X[:, 1] = [2.0, -4.0, 0.0]
    y, _ = Q.mlp_forward(theta, X)
    # row 0: h1 = (2, 0) -> h2_0 = 6 -> y = 4; row 1: h1 = (2, 4) -> h2_0 = 10 -> 6
    assert np.allclose(y, [4.0, 6.0, 4.0])
    p["b1"][0] = -5.0        # gate closes: h1_0 = 0
    y, _ = Q.mlp_forward(theta, X)
    assert np.allclose(y, [1.0, 3.0, 1.0])


def _tiny_buffer(offset=0):
    # 3 x 5:  row0 = (c0: 1, c2: 2), row1 empty, row2 = (c2: 3, c4: 1, c1: -1)
    ip = np.array([0, 2, 2, 5]) + offset
    ix = np.array([7] * offset + [0, 2, 2, 4, 1])
    vv = np.array([9.0] * offset + [1.0, 2.0, 3.0, 1.0, -1.0])
    return ip, ix, vv


@pytest.mark.parametrize("offset", [0, 3])
def test_features_of_a_hand_made_buffer(offset):
    ip, ix, vv = _tiny_buffer(offset)
    S0 = np.array([[4.0, 1.0], [1.0, 2.0]])
    f = Q.buffer_features(ip, ix, vv, 5, 2, S0, 9)
    want = np.zeros(16)
    want[0] = 1
    want[1] = math.log(3) / 10
    want[2] = math.log(5) / 20
    want[3] = math.log(5) / 15
    want[4] = 2 / 256
    want[5] = math.log(5 / 3) / 5
    want[6] = math.log(16 / 5) / 10          # ||A'||^2 = 1 + 4 + 9 + 1 + 1
    want[7] = 11 / 16                        # row norms^2 (5, 0, 11)
    want[8] = 2 / 5                          # column counts (1, 1, 2, 0, 1)
    want[9] = 7 / 25
    want[10] = 3 * (4 + 0 + 9) / 25 - 1      # row counts (2, 0, 3)
    want[11] = math.log(9) / 3
    want[12] = 22 / 36
    want[13] = 4 / 6
    want[14] = math.log(1 + 5 / 6)
    want[15] = 1 - 4 / 5
    assert np.allclose(f, want, rtol=0, atol=1e-15)


def test_features_of_an_empty_buffer():
    f = Q.buffer_features([4, 4, 4], [], [], 10, 3, np.zeros((3, 3)), 5)
    assert f[0] == 1 and f[15] == 1 and f[2] == 0 and f[12] == 0


def test_ladder_and_label_rule():
    assert Q.ladder(13) == [1, 2, 3, 4, 6, 8, 11, 13]
    assert Q.ladder(1) == [1]
    qs = [1, 2, 3, 4, 13]
    e = [90.0, 99.0, 99.95, 99.99, 100.0]
    assert Q.label(qs, e, [True] * 5, 1e-3) == 3        # 99.95 >= 99.9
    assert Q.label(qs, e, [True] * 5, 2e-2) == 2
    assert Q.label(qs, e, [True, True, False, True, True], 1e-3) == 4   # VS rejected q = 3
    assert Q.label(qs, e, [False] * 5, 1e-3) == 13


def test_predict_q_rounds_up_and_clamps():
    theta = np.zeros(Q.NPARAM)
    Q.unpack(theta)["b3"][0] = 2.2
    f = np.zeros(16)
    assert Q.predict_q(theta, f, 13, margin=1.0) == 4
    Q.unpack(theta)["b3"][0] = -7
    assert Q.predict_q(theta, f, 13) == 1
    Q.unpack(theta)["b3"][0] = 40
    assert Q.predict_q(theta, f, 13) == 13


def test_first_gram_is_the_gram_of_the_start_block():
    import scipy.sparse as sp
    from oracle import philox
    rng = np.random.default_rng(3)
    A = sp.random(40, 30, density=0.2, random_state=4, format="csr")
    S0 = Q.first_gram(A, 7, 2, 5)
    G = philox.gaussian_G(7, 2, 0, 30, 5)
    Y = A.toarray() @ G
    assert np.allclose(S0, Y.T @ Y)
    assert np.allclose(S0, S0.T)
    assert np.all(np.linalg.eigvalsh(S0) >= -1e-10)
    del rng
