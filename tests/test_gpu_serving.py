"""Continuous-batching reconstruction server on the GPU: every request's image
is the same whether it runs alone or interleaved with others, matches the
oracle's EM iterations, and the admission estimate bounds the device memory a
request really holds."""
import numpy as np
import pytest

import oracle
from paper_2301_09710_gb300.serving import GpuExecutor, Request, make_requests, serve, serve_plain

from gpu_helpers import assert_close, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _mixed(n=7, seed=11):
    # ragged sizes, PSFs and view counts; all arrive within a few milliseconds
    return make_requests(n, rate=2000.0, seed=seed, large_frac=0.0, iters=(3, 5), sizes=(24, 33, 40),
                         nzs=(7, 12, 16), views=(9, 16, 20), psfs=(3, 5, 7))


def test_same_result_alone_and_in_the_mix():
    reqs = _mixed()
    ex = GpuExecutor(n_streams=3, iters_per_step=1)
    mixed = serve(reqs, ex, mem_budget=8 << 30, max_active=4)
    ex.close()
    assert mixed.peak_active >= 2, "requests did not overlap"
    ex1 = GpuExecutor(n_streams=1, iters_per_step=3)
    alone = serve_plain(reqs, ex1)
    ex1.close()
    assert [r.rid for r in mixed.results] == [r.rid for r in alone.results] == [q.rid for q in reqs]
    for a, b in zip(mixed.results, alone.results):
        # deterministic kernels (no atomics): identical bits whatever runs beside them
        assert np.array_equal(a.x, b.x), f"request {a.rid} differs between the mix and alone"
    # and the served images are the oracle's MLEM iterates
    for q, r in zip(reqs[:3], mixed.results[:3]):
        psf = oracle.psf_from_factors(q.fx, q.fz)
        ang = oracle.default_angles(q.nview)
        s = oracle.sensitivity(q.mu, psf, q.dy, ang)
        x = q.x0.astype(np.float64)
        for _ in range(q.niter):
            x = oracle.em_step(x, q.y, q.rbar, q.mu, psf, q.dy, ang, s=s)
        assert_close(r.x, x, rel_l2=1e-5, max_rel=1e-3, what=f"served request {q.rid} vs oracle MLEM")


def test_memory_budget_limits_admission_on_the_gpu():
    reqs = _mixed(6, seed=12)
    needs = sorted(GpuExecutor.plan_bytes(q) for q in reqs)
    budget = 2 * needs[-1]
    assert sum(needs) > budget
    ex = GpuExecutor(n_streams=2, keep_images=False)
    st = serve(reqs, ex, mem_budget=budget, max_active=8)
    ex.close()
    fit = max(k for k in range(1, 7) if sum(needs[:k]) <= budget)   # most requests that fit at once
    assert len(st.results) == 6 and st.peak_bytes <= budget and st.peak_active <= fit < 6


@pytest.mark.parametrize("shape", [(24, 7, 9, 3), (33, 12, 16, 7), (64, 32, 64, 11), (128, 64, 120, 29),
                                   (192, 128, 128, 37), (128, 128, 128, 21)])
@pytest.mark.parametrize("low_memory", [False, True])
def test_plan_bytes_bounds_what_a_plan_allocates(shape, low_memory):
    from paper_2301_09710_gb300 import synthetic
    from paper_2301_09710_gb300.projector import SpectPlan, plan_bytes
    nx, nz, nv, p = shape
    _, mu, _ = synthetic.small_phantom(nx, nz, 0)
    fx, fz = synthetic.depth_psf_factors(nx, p, p, 1.0, 4.0, aniso=False)
    plan = SpectPlan(nx, nz, nv, mu=mu, fx=fx, fz=fz, low_memory=low_memory)
    held = plan.info()["device_bytes"]
    plan.close()
    bound = plan_bytes(nx, nz, nv, p, p, 1, separable=True, low_memory=low_memory)
    assert held <= bound <= 2 * held + (1 << 20), (held, bound)
    if not low_memory:
        req = Request(0, 0.0, nx, nz, nv, 1, mu, fx, fz, np.zeros((nv, nz, nx), np.float32))
        assert GpuExecutor.plan_bytes(req) >= held + 4 * (nx * nx * nz + 2 * nv * nz * nx)


def test_compact_fallback_on_the_gpu(monkeypatch):
    """A request that does not fit beside a running one is admitted with a
    compact plan (attenuation recomputed per view chunk) and its image matches
    the caching plan's within the FP32 tolerance."""
    monkeypatch.setenv("SPECT_SLAB_MB", "8")  # chunks of a few views, so compact plans are smaller
    # 64x64x32, 60 views: the attenuation of every view (31 MB) dominates the plan
    reqs = make_requests(2, rate=2000.0, seed=21, large_frac=0.0, iters=(3, 3), sizes=(64,), nzs=(32,),
                         views=(60,), psfs=(7,))
    reqs[0].niter = 24  # the first one runs long
    full = [GpuExecutor.plan_bytes(q) for q in reqs]
    small = [GpuExecutor.plan_bytes(q, compact=True) for q in reqs]
    assert small[1] < full[1]
    budget = max(full[1], full[0] + small[1])
    assert full[0] + full[1] > budget
    ex = GpuExecutor(n_streams=2, iters_per_step=1)
    st = serve(reqs, ex, mem_budget=budget, max_active=4, compact_fallback=True)
    ex.close()
    assert st.compact == 1 and st.peak_active == 2 and st.peak_bytes <= budget
    ex1 = GpuExecutor(n_streams=1, iters_per_step=3)
    alone = serve_plain(reqs, ex1)
    ex1.close()
    for a, b in zip(st.results, alone.results):
        assert_close(a.x, b.x, rel_l2=1e-5, max_rel=1e-3, what=f"request {a.rid}: compact vs caching plan")
