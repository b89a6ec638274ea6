"""GPU tests of the learned predictor: the hand-written backward kernel's
gradient against the FP64 CPU oracle, training lowers the loss, inference
picks the oracle network's masked argmin, and plans built from its choices
stay within the bound."""

import numpy as np
import pytest

from oracle import mlp_ref as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import torch
    from paper_1608_05265_gb300 import build, gbgemm
    build.build()
    hd = gbgemm.Handle(0)
    hd.set_stream(torch.cuda.current_stream())
    yield hd
    hd.close()


def synthetic_set(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, 8)).astype(np.float32)
    X[:, 3:] = (X[:, 3:] > 0.5)
    # a smooth target: which configuration is best depends on the shape features
    base = np.stack([X[:, 0] + X[:, 1] - X[:, 2], 2 * X[:, 2] - X[:, 0], X[:, 1] * X[:, 2],
                     1 - X[:, 2], 0.5 * X[:, 0] + X[:, 3], X[:, 4] + X[:, 2] * X[:, 1]], axis=1)
    y = (base - base.min(axis=1, keepdims=True)).astype(np.float32)
    M = np.ones_like(y)
    M[X[:, 2] < 0.3, 3:] = 0.0  # the split configurations are illegal for small k
    y = y * M
    return X, y, M


def test_gradient_matches_fp64_oracle(h):
    import torch
    from paper_1608_05265_gb300 import gbgemm
    rng = np.random.default_rng(7)
    theta = rng.normal(0, 0.3, gbgemm.MLP_PARAMS).astype(np.float32)
    h.predictor_set(theta)
    X, y, M = synthetic_set(8, 200)
    grad = torch.zeros(gbgemm.MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = h.predictor_loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(M).cuda(), grad)
    L, g = R.loss_grad(theta.astype(np.float64), X, y, M)
    assert abs(loss - L) <= 1e-4 * abs(L)
    gg = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - g) <= 1e-4 * np.linalg.norm(g)
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    assert np.all(np.abs(gg[big] - g[big]) <= 1e-3 * np.abs(g[big]) + 1e-6)


def test_training_lowers_loss_and_inference_matches_oracle(h):
    import torch
    from paper_1608_05265_gb300 import gbgemm, predictor
    X, y, M = synthetic_set(9, 3000)
    h2 = gbgemm.Handle(0)
    h2.set_stream(torch.cuda.current_stream())
    dx, dy, dm = (torch.from_numpy(a).cuda() for a in (X, y, M))
    l0 = h2.predictor_train(dx, dy, dm, epochs=1, lr=1e-6, seed=1)   # nearly untrained
    l1 = h2.predictor_train(dx, dy, dm, epochs=60, lr=3e-3, seed=1)
    assert l1 < 0.25 * l0
    theta = h2.predictor_get()
    legal = predictor.legal_bits(np.where(M > 0, 1.0, -1.0))
    cfg, scores = predictor.predict(h2, X, legal)
    out, _ = R.forward(theta.astype(np.float64), X)
    assert np.allclose(scores, out, rtol=1e-4, atol=1e-4)
    want = R.predict(theta.astype(np.float64), X, legal)
    # where two legal scores are within float rounding the argmin may differ
    srt = np.sort(np.where(M > 0, out, np.inf), axis=1)
    clear = (srt[:, 1] - srt[:, 0]) > 1e-4
    assert np.array_equal(cfg[clear], want[clear])
    h2.close()


def test_predicted_plan_within_bound(h):
    import torch
    from paper_1608_05265_gb300 import gbgemm
    from test_gpu_grouped import Batch, random_specs
    rng = np.random.default_rng(3)
    h.predictor_set(rng.normal(0, 0.3, gbgemm.MLP_PARAMS).astype(np.float32))
    specs = random_specs(61, 60, 16, 800, alphas=(1.0, 2.0), betas=(0.0, -0.5))
    b = Batch(specs, 61)
    plan = gbgemm.GroupedPlan(h, b.probs, config_source=gbgemm.CONFIG_PREDICTED)
    cfg = plan.configs()
    for c, (ta, tb, m, n, k, alpha, beta) in zip(cfg, specs):
        assert 0 <= c < gbgemm.NUM_CONFIGS and (c < 3 or k >= 16)
    plan.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert h.get_device_status() == 0
    b.check(nthreads=4)
    plan.close()


def test_trained_predictor_gains_over_the_default_rule(h):
    """What the trained network gains over the method without it: on 64
    held-out shapes (seed 5, never seen in training), every legal
    configuration is timed by the exhaustive tuner, and the shipped weights'
    choices must cost less, in geometric mean over the shapes, than the fixed
    default rule's; they must also be exactly the tuner's best more often."""
    import os
    from paper_1608_05265_gb300 import predictor
    if not os.path.exists(predictor.DEFAULT_WEIGHTS):
        pytest.fail("trained predictor weights are missing")
    params, _ = predictor.load_weights()
    h.predictor_set(params)
    shapes = predictor.shape_set(5, 64)
    cost, _ = predictor.label(h, shapes, reps=2)
    choice, _ = predictor.predict(h, predictor.features(shapes), predictor.legal_bits(cost))
    assert np.all(cost[np.arange(len(shapes)), choice] > 0)  # only legal configurations are chosen
    learned = predictor.regret(cost, choice)
    default = predictor.regret(cost, predictor.default_choice(shapes))
    assert learned["geomean_ratio"] < default["geomean_ratio"], (learned, default)
    assert learned["exact"] > default["exact"], (learned, default)
