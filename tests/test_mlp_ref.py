"""Pins of the predictor network's CPU oracle: its analytic gradient against
central finite differences of its loss (an independent computation), a
closed form for a one-hot output, and the masked argmin."""

import numpy as np

from oracle import mlp_ref as R


def rand_case(seed, n=23):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.4, R.N_PARAMS)
    X = rng.uniform(0, 1, (n, R.N_IN))
    Y = rng.normal(0, 1, (n, R.N_OUT))
    M = (rng.uniform(0, 1, (n, R.N_OUT)) < 0.7).astype(np.float64)
    return theta, X, Y, M


def test_param_count_matches_layout():
    assert R.N_PARAMS == 8 * 64 + 64 + 64 * 64 + 64 + 6 * 64 + 6 == 5126


def test_gradient_matches_central_differences():
    theta, X, Y, M = rand_case(0)
    L, g = R.loss_grad(theta, X, Y, M)
    assert abs(L - R.loss(theta, X, Y, M)) < 1e-12
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(R.N_PARAMS, 300, replace=False), np.arange(5120, 5126), np.arange(0, 8)])
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (R.loss(tp, X, Y, M) - R.loss(tm, X, Y, M)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_output_bias_gradient_closed_form():
    # dL/db3[c] = 2 sum_s mask[s,c] (out[s,c] - y[s,c]) / sum mask
    theta, X, Y, M = rand_case(2)
    out, _ = R.forward(theta, X)
    _, g = R.loss_grad(theta, X, Y, M)
    want = 2 * ((out - Y) * M).sum(0) / M.sum()
    assert np.allclose(g[-6:], want, rtol=1e-12, atol=1e-14)


def test_masked_argmin():
    theta, X, _, _ = rand_case(3, n=50)
    out, _ = R.forward(theta, X)
    legal = np.full(50, 0b111111)
    legal[::3] = 0b000111
    legal[5] = 0
    got = R.predict(theta, X, legal)
    for s in range(50):
        if legal[s] == 0:
            assert got[s] == -1
            continue
        cand = [c for c in range(6) if (legal[s] >> c) & 1]
        assert got[s] == cand[int(np.argmin(out[s, cand]))]


def hand_network():
    """A hand-set network with a few nonzero weights (row = output unit)."""
    p = {name: np.zeros(shape) for name, shape in R.SIZES}
    p["W1"][0, 0], p["W1"][0, 1], p["b1"][0] = 1.0, -2.0, 0.5   # z1[0] = x0 - 2 x1 + 0.5
    p["W1"][1, 2], p["b1"][1] = 3.0, -1.0                       # z1[1] = 3 x2 - 1
    p["W1"][2, 0] = -1.0                                        # z1[2] = -x0 (cut by the ReLU)
    p["W2"][0, 0], p["W2"][0, 1], p["b2"][0] = 2.0, 1.0, -0.25  # z2[0] = 2 h1[0] + h1[1] - 0.25
    p["W2"][1, 2], p["b2"][1] = 5.0, 0.75                       # z2[1] = 5 h1[2] + 0.75
    p["W2"][2, 0] = -1.0                                        # z2[2] = -h1[0] (cut by the ReLU)
    p["W3"][0, 0], p["W3"][0, 1], p["b3"][0] = 1.0, 2.0, 0.125  # out0 = h2[0] + 2 h2[1] + 1/8
    p["W3"][1, 0] = -1.0                                        # out1 = -h2[0] (no ReLU on the output)
    p["W3"][2, 2], p["b3"][2] = 4.0, -0.5                       # out2 = 4 h2[2] - 1/2
    p["W3"][3, 1] = 1.0                                         # out3 = h2[1]
    p["b3"][5] = 3.0                                            # out5 = 3
    return R.pack(p)


def test_forward_of_a_hand_set_network():
    # Worked by hand.  Row 1, x = (1, 1/4, 2, 0 ...): z1 = (1, 5, -1) -> h1 = (1, 5, 0);
    # z2 = (6.75, 0.75, -1) -> h2 = (6.75, 0.75, 0); out = (8.375, -6.75, -0.5, 0.75, 0, 3).
    # Row 2, x = (0, 0, 1/2, 0 ...): h1 = (0.5, 0.5, 0); h2 = (1.25, 0.75, 0);
    # out = (2.875, -1.25, -0.5, 0.75, 0, 3).
    # A dropped b2 changes out0 and out3, a missing hidden ReLU changes out2,
    # a ReLU on the output changes out1, a transposed W1 changes every row.
    theta = hand_network()
    X = np.zeros((2, 8))
    X[0, :3] = (1.0, 0.25, 2.0)
    X[1, 2] = 0.5
    out, (_, z1, h1, z2, h2) = R.forward(theta, X)
    assert np.array_equal(out, [[8.375, -6.75, -0.5, 0.75, 0.0, 3.0], [2.875, -1.25, -0.5, 0.75, 0.0, 3.0]])
    assert np.array_equal(h1[:, :3], [[1.0, 5.0, 0.0], [0.5, 0.5, 0.0]])
    assert np.array_equal(h2[:, :3], [[6.75, 0.75, 0.0], [1.25, 0.75, 0.0]])
    # the parameter layout: W1 is 64 x 8 row-major, first in the flat vector
    assert theta[1] == -2.0 and theta[8 + 2] == 3.0 and theta[64 * 8] == 0.5
    # loss by hand with y = 0 and the mask keeping out0 and out1 of row 1 only:
    # (8.375^2 + 6.75^2) / 2
    M = np.zeros((2, 6))
    M[0, :2] = 1.0
    assert R.loss(theta, X, np.zeros((2, 6)), M) == (8.375 ** 2 + 6.75 ** 2) / 2
    assert list(R.predict(theta, X, np.array([0b111111, 0b111100]))) == [1, 2]


def test_schedule_network_layout_and_hand_forward():
    # The schedule network: the same hidden layers, 39 outputs (7271 parameters).
    # The hand network's first six output rows placed in a 39-output vector
    # give the same six outputs by hand; output 38 = b3[38] = -2 and output
    # 20 = 2 h2[1] are set here, and the argmin over bits of a 39-bit mask.
    p6 = R.unpack(hand_network())
    p = {name: np.zeros(shape) for name, shape in R.sizes(39)}
    for name in ("W1", "b1", "W2", "b2"):
        p[name] = p6[name].copy()
    p["W3"][:6] = p6["W3"]
    p["b3"][:6] = p6["b3"]
    p["W3"][20, 1] = 2.0
    p["b3"][38] = -2.0
    theta = R.pack(p)
    assert theta.size == 7271 == R.N_HIDDEN_PARAMS + 39 * 65
    assert R.n_outputs(theta) == 39
    X = np.zeros((2, 8))
    X[0, :3] = (1.0, 0.25, 2.0)
    X[1, 2] = 0.5
    out, _ = R.forward(theta, X)
    assert out.shape == (2, 39)
    assert np.array_equal(out[:, :6], [[8.375, -6.75, -0.5, 0.75, 0.0, 3.0], [2.875, -1.25, -0.5, 0.75, 0.0, 3.0]])
    assert out[0, 20] == 1.5 and out[1, 20] == 1.5 and out[0, 38] == -2.0
    full = (1 << 39) - 1
    assert list(R.predict(theta, X, [full, full & ~(1 << 1) & ~(1 << 38)])) == [1, 2]
    assert list(R.predict(theta, X, [1 << 38, 0])) == [38, -1]


def test_schedule_network_gradient_matches_central_differences():
    rng = np.random.default_rng(7)
    n_par = R.N_HIDDEN_PARAMS + 39 * 65
    theta = rng.normal(0, 0.4, n_par)
    X = rng.uniform(0, 1, (17, R.N_IN))
    Y = rng.normal(0, 1, (17, 39))
    M = (rng.uniform(0, 1, (17, 39)) < 0.5).astype(np.float64)
    L, g = R.loss_grad(theta, X, Y, M)
    idx = np.concatenate([rng.choice(n_par, 200, replace=False), np.arange(n_par - 39, n_par)])
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (R.loss(tp, X, Y, M) - R.loss(tm, X, Y, M)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])
