"""Plans that recompute the Eq. (1) attenuation per view chunk
(SPECT_PLAN_RECOMPUTE_ATTENUATION) against plans that cache it for every view.

* A x, A' y and EM iterates are bitwise those of the caching plan when both
  take the same adjoint passes (the view sum of A' is chunked the same way),
  with the views spread over several ragged chunks, and they match the oracle;
* the plan allocates less than the caching plan and stays within its
  spect_plan_bytes bound;
* launch shapes and the autotuner work on such plans; they run in a batch;
* the mode is refused where it does not apply.
"""
import numpy as np
import pytest

import oracle
from paper_2301_09710_gb300 import synthetic

from gpu_helpers import assert_close, dev, host, make_plan, need_gpu, oracle_psf, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _plan(prob, ang, recompute, **kw):
    from paper_2301_09710_gb300 import SpectPlan
    nz, ny, nx = prob.x.shape
    return SpectPlan(nx, nz, len(ang), mu=prob.mu, dy=prob.dy, fx=prob.fx, fz=prob.fz, angles=ang,
                     recompute_attenuation=recompute, **kw)


def _run(plan, prob, y, rbar, x0):
    v = host(plan.forward(dev(prob.x)))
    b = host(plan.back(dev(y)))
    xe = dev(x0)
    plan.em_step(xe, dev(y), dev(rbar), niter=2)
    return v, b, host(xe)


# nx, nz, nview, psf
CASES = [(40, 12, 10, 9), (33, 20, 7, 21), (48, 16, 13, 37), (64, 36, 6, 5)]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}v{c[2]}p{c[3]}" for c in CASES])
def test_recomputing_plan_is_bitwise_the_caching_plan(case, monkeypatch):
    nx, nz, nv, p = case
    # a 1 MiB budget spreads the views over several chunks (the last one
    # ragged); both plans take the adjoint one view per pass, so their view
    # sums of A' round the same way whatever chunk each plan chose
    monkeypatch.setenv("SPECT_SLAB_MB", "1")
    monkeypatch.setenv("SPECT_ADJ_CHUNK", "1")
    prob = synthetic.config1(seed=nx + p, nx=nx, nz=nz, nview=nv, psf_size=p)
    ang = oracle.default_angles(nv)
    psf = oracle_psf(prob, "fused")
    ybar = oracle.forward(prob.x, prob.mu, psf, prob.dy, ang)
    y = synthetic.poisson_counts(ybar * 20, 1)
    rbar = np.full_like(y, 0.1 * float(y.mean()) + 0.01)
    x0 = np.where(prob.body, 1.0, 0.0).astype(np.float32) + 0.05
    cached = _plan(prob, ang, False)
    plan = _plan(prob, ang, True)
    assert plan.info()["view_chunk"] < nv, "the budget should split the views into chunks"
    got = _run(plan, prob, y, rbar, x0)
    want = _run(cached, prob, y, rbar, x0)
    for g, w, what in zip(got, want, ("A x", "A' y", "EM iterates")):
        assert np.array_equal(g, w), f"{what}: recomputing plan differs from the caching plan"
    assert_close(got[0], ybar, what="A x, recomputed attenuation")
    assert_close(got[1], oracle.back(y, prob.mu, psf, prob.dy, ang), what="A' y, recomputed attenuation")
    plan.check()
    cached.check()
    plan.close()
    cached.close()


def test_recomputing_plan_memory_and_bound():
    from paper_2301_09710_gb300.projector import plan_bytes
    prob = synthetic.config2(seed=0)
    ang = oracle.default_angles(128)
    # 128 views: the caching plan holds every view's factors, the recomputing one a chunk's
    full_cache = plan_bytes(128, 80, 128, 37, 37)
    bound = plan_bytes(128, 80, 128, 37, 37, recompute_attenuation=True)
    assert bound < full_cache / 2, (bound, full_cache)
    plan = _plan(prob, ang, True)
    cached = _plan(prob, ang, False)
    assert plan.info()["device_bytes"] <= bound
    assert plan.info()["view_chunk"] < 128
    assert plan.info()["device_bytes"] < cached.info()["device_bytes"] / 2
    x = dev(prob.x)
    assert np.array_equal(host(plan.forward(x)), host(cached.forward(x)))
    plan.check()
    plan.close()
    cached.close()
    # against the oracle on 16 of the views (one chunk)
    ang16 = ang[::8]
    plan = _plan(prob, ang16, True)
    assert_close(host(plan.forward(x)), oracle.forward(prob.x, prob.mu, oracle_psf(prob, "fused"), prob.dy, ang16),
                 what="A x at 128x128x80, 37x37 PSF, recomputed attenuation")
    plan.check()
    plan.close()


def test_recomputing_plan_launch_shapes_autotune_and_batch(monkeypatch):
    from paper_2301_09710_gb300 import SpectBatch
    monkeypatch.setenv("SPECT_SLAB_MB", "1")
    prob = synthetic.config1(seed=5, nx=48, nz=16, nview=9, psf_size=11)
    ang = oracle.default_angles(9)
    psf = oracle_psf(prob, "fused")
    want = oracle.forward(prob.x, prob.mu, psf, prob.dy, ang)
    plan = _plan(prob, ang, True)
    x = dev(prob.x)
    for J, aJ, tiles in ((4, 8, 1), (16, 4, 2), (8, 8, 3)):
        plan.set_tuning(J, aJ, tiles)
        assert_close(host(plan.forward(x)), want, what=f"A x, shape {plan.tuning}")
    plan.autotune()
    assert_close(host(plan.forward(x)), want, what=f"A x, autotuned {plan.tuning}")
    y = synthetic.poisson_counts(want * 20, 2)
    x0 = np.where(prob.body, 1.0, 0.0).astype(np.float32) + 0.05
    alone = dev(x0)
    plan.em_step(alone, dev(y), None, niter=2)
    other = make_plan(synthetic.config1(seed=6, nx=24, nz=8, nview=5, psf_size=5), oracle.default_angles(5), "fused")
    yo = dev(np.ones((5, 8, 24), np.float32))
    batch = SpectBatch([plan, other])
    xs = [dev(x0), dev(np.ones((8, 24, 24), np.float32))]
    batch.em_step(xs, [dev(y), yo], None, niter=2)
    assert np.array_equal(host(xs[0]), host(alone)), "recomputing plan in a batch differs from the plan alone"
    batch.close()
    plan.check()
    plan.close()
    other.close()


def test_recompute_refused_where_it_does_not_apply():
    from paper_2301_09710_gb300._lib import SpectError
    prob = synthetic.config1(seed=3, nx=24, nz=8, nview=4, psf_size=5)
    ang = oracle.default_angles(4)
    with pytest.raises(SpectError):
        _plan(prob, ang, True, low_memory=True)
    with pytest.raises(SpectError):
        _plan(prob, ang, True, rotation="3pass")
