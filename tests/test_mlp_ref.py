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
