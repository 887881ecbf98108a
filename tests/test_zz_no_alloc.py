"""spect_forward_static: the forward projection for callers that cannot
allocate device memory (hosts whose device memory is reserved up front,
plug-ins whose host application owns the allocator).  Its work slab lives in a
fixed-size static device array shared by every call, so it must give the same
projections as the plan-based spect_forward, call after call, and those must
match the FP64 oracle.  This file is collected last so that a failure here
leaves every other test already run.
"""
import numpy as np
import pytest

import oracle
from paper_2301_09710_gb300 import synthetic

from gpu_helpers import assert_close, dev, host, make_plan, need_gpu, torch

pytestmark = pytest.mark.gpu


def test_static_forward_matches_plan_forward_on_consecutive_calls():
    need_gpu()
    from paper_2301_09710_gb300.projector import forward_static

    prob = synthetic.config1(seed=4, nx=64, nz=32, nview=24, psf_size=11)
    ang = oracle.default_angles(prob.nview)
    plan = make_plan(prob, ang, "fused")
    x = dev(prob.x)
    v_ref = host(plan.forward(x))
    plan.check()
    mu, fx, fz = dev(prob.mu), dev(prob.fx), dev(prob.fz)
    v_o = oracle.forward(prob.x, prob.mu, oracle.psf_from_factors(prob.fx, prob.fz), prob.dy, ang)
    for _ in range(2):
        out = torch.full(plan.proj_shape, float("nan"), device="cuda")
        forward_static(x, prob.nview, fx, fz, mu=mu, dy=prob.dy, angles=ang, out=out)
        got = host(out)
        assert_close(got, v_ref, what="static-scratch forward vs plan forward")
        assert_close(got, v_o, what="static-scratch forward vs FP64 oracle")


def test_static_forward_rejects_volume_beyond_scratch():
    need_gpu()
    from paper_2301_09710_gb300 import _lib
    from paper_2301_09710_gb300.projector import forward_static

    x = torch.zeros((129, 256, 256), device="cuda")  # 8,454,144 voxels > 8 Mi
    f = torch.ones((1, 256, 1), device="cuda")
    with pytest.raises(_lib.SpectError, match="static scratch"):
        forward_static(x, 4, f, f.clone())
