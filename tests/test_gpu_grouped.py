"""GPU parity of the grouped sgemm: every problem of a batch against the FP64
oracle under the acceptance bound, graph replays, skipped and degenerate
problems, bad plans."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1608_05265_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import torch
    from paper_1608_05265_gb300 import build, gbgemm
    build.build()
    assert torch.cuda.is_available()
    hd = gbgemm.Handle(0)
    hd.set_stream(torch.cuda.current_stream())
    yield hd
    hd.close()


class Batch:
    """Host data, device buffers and gbgemm_problem structs of a batch."""

    def __init__(self, specs, seed):
        import torch
        from paper_1608_05265_gb300 import gbgemm
        self.specs = specs
        self.host, self.dev, self.probs = [], [], []
        for g, (ta, tb, m, n, k, alpha, beta) in enumerate(specs):
            A, lda, B, ldb, C, ldc = synth.grouped_problem_data(seed, g, ta, tb, m, n, k)
            dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C))
            self.host.append((A, lda, B, ldb, C, ldc))
            self.dev.append((dA, dB, dC))
            self.probs.append(gbgemm.problem(ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc))

    def results(self):
        return [d[2].cpu().numpy() for d in self.dev]

    def reset_c(self):
        import torch
        for (A, lda, B, ldb, C, ldc), d in zip(self.host, self.dev):
            d[2].copy_(torch.from_numpy(C))

    def check(self, outs=None, max_ratio=1.0, nthreads=0):
        outs = outs if outs is not None else self.results()
        worst = 0.0
        for (ta, tb, m, n, k, alpha, beta), (A, lda, B, ldb, C, ldc), out in zip(self.specs, self.host, outs):
            assert synth.padding_is_sentinel(out, m, n, ldc)
            if m == 0 or n == 0:
                assert np.array_equal(out.view(np.uint32), C.view(np.uint32))
                continue
            c64, bnd = O.gemm_f64(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nthreads=nthreads)
            r = O.error_ratio(synth.logical(out, m, n, ldc), c64, bnd)
            assert r <= max_ratio, (ta, tb, m, n, k, alpha, beta, r)
            worst = max(worst, r)
        return worst


def random_specs(seed, count, lo, hi, alphas=(1.0,), betas=(0.0,)):
    shapes = synth.grouped_shapes(seed, count, lo, hi)
    return [(ta, tb, m, n, k, alphas[g % len(alphas)], betas[g % len(betas)])
            for g, (ta, tb, m, n, k) in enumerate(shapes)]


def run_plan(h, batch, **kw):
    import torch
    from paper_1608_05265_gb300 import gbgemm
    plan = gbgemm.GroupedPlan(h, batch.probs, **kw)
    plan.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert h.get_device_status() == 0
    return plan


def test_grouped_default_configs(h):
    specs = random_specs(31, 160, 4, 600, alphas=(1.0, -1.5, 0.5), betas=(0.0, 1.0, -0.25))
    b = Batch(specs, 31)
    plan = run_plan(h, b)
    cfg = plan.configs()
    assert any(c >= 3 for c in cfg) and any(0 <= c < 3 for c in cfg)
    b.check(nthreads=4)
    plan.close()


def test_grouped_every_config(h):
    from paper_1608_05265_gb300 import gbgemm
    specs = random_specs(32, 120, 16, 700, alphas=(1.0, 2.0), betas=(0.0, 0.5))
    b = Batch(specs, 32)
    configs = []
    for g, (ta, tb, m, n, k, alpha, beta) in enumerate(specs):
        legal = [0, 1, 2] + ([3, 4, 5] if k >= 16 else [])
        configs.append(legal[g % len(legal)])
    plan = run_plan(h, b, configs=configs)
    assert plan.configs() == configs
    st = plan.stats()
    assert st["n_split"] + st["n_simt"] == len(specs)
    b.check(nthreads=4)
    plan.close()
    del gbgemm


def test_grouped_replay_is_deterministic_and_reuses_buffers(h):
    import torch
    specs = random_specs(33, 90, 16, 500)
    b = Batch(specs, 33)
    plan = run_plan(h, b)
    first = b.results()
    for d in b.dev:
        d[2].fill_(float("nan"))  # beta = 0: C is not read; the replay rewrites it
    plan.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    second = b.results()
    for x, y, (ta, tb, m, n, k, alpha, beta), (A, lda, B, ldb, C, ldc) in zip(first, second, specs, b.host):
        assert np.array_equal(synth.logical(x, m, n, ldc).view(np.uint32), synth.logical(y, m, n, ldc).view(np.uint32))
    b.check(first, nthreads=4)
    plan.close()


def test_grouped_degenerate_problems(h):
    import torch
    from paper_1608_05265_gb300 import gbgemm
    specs = [("N", "N", 0, 40, 200, 1.0, 0.0), ("T", "N", 40, 0, 200, 1.0, 0.0),
             ("N", "T", 64, 70, 0, 1.0, -2.0), ("N", "N", 64, 70, 300, 0.0, 0.5),
             ("T", "T", 33, 21, 150, 0.0, 1.0), ("N", "N", 130, 260, 256, 1.5, -0.25),
             ("T", "N", 17, 300, 5, 1.0, 0.0)]
    b = Batch(specs, 34)
    # alpha == 0: A and B are not read, so null pointers are allowed
    b.probs[3].A = None
    b.probs[3].B = None
    plan = run_plan(h, b)
    cfg = plan.configs()
    assert cfg[0] == -1 and cfg[1] == -1 and cfg[4] == -1
    b.check()
    plan.close()
    del torch, gbgemm


def test_grouped_bad_plans(h):
    from paper_1608_05265_gb300 import gbgemm
    specs = random_specs(35, 6, 16, 200)
    b = Batch(specs, 35)
    probs = list(b.probs)
    probs[3] = gbgemm.problem("X", "N", 4, 4, 4, 1.0, b.dev[3][0], 4, b.dev[3][1], 4, 0.0, b.dev[3][2], 4)
    rc, bad = gbgemm.create_plan_status(h, probs)
    assert rc == gbgemm.ERR_BAD_PLAN and bad == 3
    probs = list(b.probs)
    p = probs[2]
    probs[2] = gbgemm.problem(p.transa.decode(), p.transb.decode(), p.m, p.n, p.k, 1.0, p.A, 0, p.B, p.ldb, 0.0,
                              p.C, p.ldc)
    rc, bad = gbgemm.create_plan_status(h, probs)
    assert rc == gbgemm.ERR_BAD_PLAN and bad == 2
    # a split configuration for a problem with k < 16 is illegal
    small = [("N", "N", 40, 40, 12, 1.0, 0.0)]
    b2 = Batch(small, 36)
    rc, bad = gbgemm.create_plan_status(h, b2.probs, configs=[gbgemm.CFG_SPLIT_BN128])
    assert rc == gbgemm.ERR_BAD_PLAN and bad == 0


def test_grouped_uneven_batch_4096(h):
    """The uneven batch: 4096 problems, m, n, k log-uniform in [16, 1024], random
    transposes, tight leading dimensions, uniform data, alpha 1, beta 0 (seed 3);
    every problem checked against the oracle."""
    shapes = synth.grouped_shapes(3, 4096)
    specs = [(ta, tb, m, n, k, 1.0, 0.0) for (ta, tb, m, n, k) in shapes]
    b = Batch(specs, 3)
    plan = run_plan(h, b)
    st = plan.stats()
    assert st["n_split"] == 4096 and st["n_simt"] == 0  # every k >= 16: the split path
    b.check()
    plan.close()


SCALED_SHORT_K = [("N", "N", 300, 200, 256, 1.0, 0.5), ("T", "N", 200, 300, 384, 1.0, 0.0),
                  ("N", "T", 130, 129, 200, -1.0, 1.0), ("T", "T", 64, 64, 128, 2.0, 0.0)]
# k >= 512: two-part panels (three products)
SCALED_LONG_K = [("N", "N", 300, 200, 600, 1.0, 0.5), ("T", "N", 200, 300, 777, 1.0, 0.0),
                 ("N", "T", 130, 129, 512, -1.0, 1.0), ("T", "T", 64, 64, 1000, 2.0, 0.0),
                 ("N", "N", 257, 40, 530, 1.0, 0.0)]


@pytest.mark.parametrize("specs", [SCALED_SHORT_K, SCALED_LONG_K], ids=["short_k", "long_k"])
def test_grouped_badly_scaled_rows_take_the_fallback(h, specs):
    """Problems whose rows of op(A) or columns of op(B) are badly scaled (max
    |x| outside [2^-48, 2^48)): the grouped re-pack scales them by powers of
    two, in three-part (k < 512) and two-part panels alike; every result
    stays within the bound."""
    import torch
    from paper_1608_05265_gb300 import gbgemm
    b = Batch(specs, 81)
    # scale some stored rows of A by 2^60 and some of B by 2^-70
    for g, (ta, tb, m, n, k, alpha, beta) in enumerate(specs):
        A, lda, B, ldb, C, ldc = b.host[g]
        ar, ac = synth.op_shape(ta, m, k)
        br, bc = synth.op_shape(tb, k, n)
        A = A.copy(); B = B.copy()
        La = A[: lda * ac].reshape(ac, lda)
        La[:, 3:ar:17] *= np.float32(2.0**60)
        Lb = B[: ldb * bc].reshape(bc, ldb)
        Lb[1:bc:23, :br] *= np.float32(2.0**-70)
        b.host[g] = (A, lda, B, ldb, C, ldc)
        b.dev[g][0].copy_(torch.from_numpy(A))
        b.dev[g][1].copy_(torch.from_numpy(B))
    for cfg in (gbgemm.CFG_SPLIT_BN64, gbgemm.CFG_SPLIT_BN128):
        b.reset_c()
        plan = gbgemm.GroupedPlan(h, b.probs, configs=[cfg] * len(specs))
        plan.run(torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert h.get_device_status() == 0
        b.check()
        plan.close()


def test_grouped_long_k_infinities(h):
    """An infinity in op(A) on the long-k split path.  Its lo part is zero,
    but inf * hi(b) + inf * lo(b) is NaN wherever lo(b) has the other sign,
    so the split can only promise that the row it touches is non-finite (as
    the FP64 result is); every other entry stays within the bound."""
    import torch
    from paper_1608_05265_gb300 import gbgemm
    specs = [("N", "N", 150, 140, 640, 1.0, 0.0), ("T", "N", 90, 200, 520, 1.0, 0.0)]
    b = Batch(specs, 82)
    hits = []
    for g, (ta, tb, m, n, k, alpha, beta) in enumerate(specs):
        A, lda, B, ldb, C, ldc = b.host[g]
        A = A.copy()
        i, p = 7 + 11 * g, 300 + g
        A[(i + p * lda) if ta == "N" else (p + i * lda)] = np.float32(np.inf)
        b.host[g] = (A, lda, B, ldb, C, ldc)
        b.dev[g][0].copy_(torch.from_numpy(A))
        hits.append(i)
    plan = gbgemm.GroupedPlan(h, b.probs, configs=[gbgemm.CFG_SPLIT_BN128] * len(specs))
    plan.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert h.get_device_status() == 0
    for g, ((ta, tb, m, n, k, alpha, beta), (A, lda, B, ldb, C, ldc), out) in enumerate(
            zip(specs, b.host, b.results())):
        c64, bnd = O.gemm_f64(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc)
        got = synth.logical(out, m, n, ldc)
        row = hits[g]
        assert not np.any(np.isfinite(c64[row])) and not np.any(np.isfinite(got[row]))
        others = np.ones(m, bool)
        others[row] = False
        assert O.error_ratio(got[others], c64[others], bnd[others]) <= 1.0
    plan.close()
