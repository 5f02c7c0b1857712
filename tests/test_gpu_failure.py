"""Failure detection on the device without a fault: a bounded wait that runs
out latches a status the host reads, and the context stays usable."""
import time

import pytest

from gpu_util import assert_same, gpu_filter_fixed, oracle_fixed, torch_cuda
from paper_1910_09020_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    torch_cuda()
    f = binding.Filter(0)
    yield f
    f.close()


def test_bounded_wait_gives_up_and_reports(F):
    t0 = time.perf_counter()
    F.check_wait_timeout(50_000_000)  # 50 ms on a barrier nothing completes
    with pytest.raises(binding.SSError) as ei:
        F.sync()
    elapsed = time.perf_counter() - t0
    assert ei.value.code == binding.SS_ERR_TIMEOUT
    assert 0.04 < elapsed < 10.0
    F.sync()  # the status was cleared
    reads, refs = synth.pairs_fixed(8, 0, 3000, 100, synth.SHORT_POISSON)
    acc, obs = gpu_filter_fixed(F, reads, refs, 4)
    oacc, oobs = oracle_fixed(reads, refs, 4)
    assert_same(acc, obs, oacc, oobs, "after a timed-out wait")


def test_bounded_wait_rejects_bad_limits(F):
    for bad in (0, 999, 10_000_000_001):
        with pytest.raises(binding.SSError) as ei:
            F.check_wait_timeout(bad)
        assert ei.value.code == binding.SS_ERR_INVALID_ARG
