"""Failure detection on the GPU without a fault: a bounded device wait that
nothing completes runs out, the kernel records SPECT_ETIMEOUT in the plan's
error word and returns; the host reads it with check(), and the plan (and the
CUDA context) stay usable."""
import numpy as np
import pytest

import oracle
from paper_2301_09710_gb300 import synthetic

from gpu_helpers import assert_close, dev, host, make_plan, need_gpu, oracle_psf, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("use_stream_check", [False, True])
def test_bounded_wait_runs_out_and_is_reported(use_stream_check):
    from paper_2301_09710_gb300._lib import SpectError
    prob = synthetic.config1(seed=3, nx=24, nz=8, nview=6, psf_size=5)
    ang = oracle.default_angles(6)
    plan = make_plan(prob, ang, "fused")
    st = torch.cuda.current_stream()
    plan.check()
    plan.selftest_timeout(1 << 22, stream=st)  # about 2 ms of spinning, then the wait gives up
    with pytest.raises(SpectError) as e:
        plan.check(stream=st) if use_stream_check else plan.check()
    assert "SPECT_ETIMEOUT" in str(e.value)
    plan.check()  # the error word was cleared
    # the plan and the context still work
    v = host(plan.forward(dev(prob.x)))
    assert_close(v, oracle.forward(prob.x, prob.mu, oracle_psf(prob, "fused"), prob.dy, ang), what="A x after timeout")
    plan.check()
    plan.close()
