"""Failure detection on the GPU, in the form that faults nothing: a bounded
mbarrier wait that nothing completes runs out after 1 ms, the kernel records
GBGEMM_ERR_DEVICE_TIMEOUT in the device status word and returns normally; the
host reads the status, the read clears it, and the same handle then computes
oracle-correct results on both paths."""

import pytest

from paper_1608_05265_gb300 import synth

from gpu_util import SIMT, SPLIT, check_full

pytestmark = pytest.mark.gpu


def test_expired_wait_is_reported_and_the_context_stays_usable():
    import torch
    from paper_1608_05265_gb300 import build, gbgemm
    build.build()
    h = gbgemm.Handle(0)
    h.set_stream(torch.cuda.current_stream())
    assert h.get_device_status() == 0
    L = gbgemm.lib()  # out-of-range limits are refused
    assert L.gbgemm_debug_expire_wait(h._h, 0) == gbgemm.ERR_INVALID_VALUE
    assert L.gbgemm_debug_expire_wait(h._h, 100000001) == gbgemm.ERR_INVALID_VALUE
    h.debug_expire_wait(1_000_000)
    assert h.get_device_status() == gbgemm.ERR_DEVICE_TIMEOUT
    assert h.get_device_status() == 0  # reading cleared it
    m, n, k = 300, 260, 640
    A, lda, B, ldb, C, ldc = synth.gemm_problem("uniform", 91, "N", "T", m, n, k, pad=3)
    for path in (SPLIT, SIMT):
        check_full(h, path, "N", "T", m, n, k, 1.5, A, lda, B, ldb, -0.25, C, ldc)
    # twice in a row: each expiry is reported on its own
    h.debug_expire_wait(1_000_000)
    h.debug_expire_wait(2_000_000)
    assert h.get_device_status() == gbgemm.ERR_DEVICE_TIMEOUT
    assert h.get_device_status() == 0
    h.close()
