"""Failure detection on the GPU without a GPU fault.

The scorers wait for their TMA window copies on an mbarrier with a bounded,
timer-limited wait, and in the persistent form a CTA waits, bounded the same
way, for the task it claimed to be published.  The self-test entry points
run those waits on an mbarrier that nothing completes (no copy is issued)
and on a task flag that nothing sets: each wait must give up after its
limit, the give-up must reach the host as SAM_ERR_TIMEOUT through the
scorers' device error flag (cleared on read), and the context must stay
usable: a detection right after it returns the usual result.
"""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2112_05576_gb300 as sam  # noqa: E402
from paper_2112_05576_gb300.sam import SAM_ERR_ARG, SAM_ERR_TIMEOUT  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sam.lib()


def test_bounded_wait_gives_up_and_reports_timeout():
    tm, sc, truth = synth.config1_scene()
    m = sam.Model(tm, 30, 60, 3, 1.0)
    p = sam.default_detect_params(min_score=0.7)
    before = sam.detect(m, torch.from_numpy(sc).cuda(), p)
    for test in (sam.selftest_wait_timeout, sam.selftest_task_wait_timeout):
        for limit_us in (500, 3000):
            status, ms = test(limit_us)
            assert status == SAM_ERR_TIMEOUT
            assert limit_us * 1e-3 <= ms < limit_us * 1e-3 + 50.0
            assert sam.take_device_error() == 0          # the flag was read and cleared
    after = sam.detect(m, torch.from_numpy(sc).cuda(), p)
    assert [(d["x"], d["y"], d["k"]) for d in after] == [(d["x"], d["y"], d["k"]) for d in before]
    assert len(after) == len(truth)


def test_selftest_rejects_bad_limits():
    for bad in (0, -5, 2_000_000):
        for test in (sam.selftest_wait_timeout, sam.selftest_task_wait_timeout):
            status, _ = test(bad)
            assert status == SAM_ERR_ARG
