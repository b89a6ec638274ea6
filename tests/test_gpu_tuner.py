"""GPU tests of the autotuner: it times exactly the legal configurations,
its choice is the argmin of what it measured, its cache survives a save and
load, and plans and calls built from its choices stay oracle-exact within
the bound."""

import numpy as np
import pytest

from paper_1608_05265_gb300 import synth

from gpu_util import check_full

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


def test_tuner_times_legal_configs_only(h):
    from paper_1608_05265_gb300 import gbgemm, predictor
    for shape in [("N", "N", 300, 200, 64, 1, 1, 1), ("T", "N", 1000, 700, 512, 0, 1, 0), ("N", "T", 20, 4000, 300, 1, 0, 1)]:
        lat, cost, bl, bc = h.autotune(predictor.tuning_problem(shape), reps=2)
        k = shape[4]
        for c in range(gbgemm.NUM_CONFIGS):
            legal = c < 3 or k >= 16
            assert (lat[c] > 0) == legal and (cost[c] > 0) == legal
        assert bl == int(np.argmin([x if x > 0 else np.inf for x in lat]))
        assert bc == int(np.argmin([x if x > 0 else np.inf for x in cost]))


def test_tuning_cache_roundtrip(h, tmp_path):
    from paper_1608_05265_gb300 import predictor
    p = predictor.tuning_problem(("N", "T", 333, 444, 256, 1, 1, 1))
    first = h.autotune(p)
    path = str(tmp_path / "cache.txt")
    h.tuning_save(path)
    h.tuning_clear()
    h.tuning_load(path)
    again = h.autotune(p)  # served from the loaded cache
    assert np.allclose(first[0], again[0], rtol=1e-4) and first[2:] == again[2:]


def test_tuned_single_sgemm_and_grouped_plan(h):
    import torch
    from paper_1608_05265_gb300 import gbgemm
    h.set_tuning(1)
    try:
        for (ta, tb, m, n, k) in [("N", "N", 700, 500, 300), ("T", "T", 129, 1000, 96)]:
            A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 51, ta, tb, m, n, k, pad=3)
            check_full(h, gbgemm.PATH_AUTO, ta, tb, m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc)
    finally:
        h.set_tuning(0)
    # a grouped plan whose configurations come from the tuner
    from test_gpu_grouped import Batch, random_specs
    specs = random_specs(52, 40, 16, 700, alphas=(1.0,), betas=(0.0, 0.5))
    b = Batch(specs, 52)
    plan = gbgemm.GroupedPlan(h, b.probs, config_source=gbgemm.CONFIG_TUNED)
    plan.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert h.get_device_status() == 0
    b.check(nthreads=4)
    plan.close()
