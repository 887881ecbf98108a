"""Parity at the paper-scale workload (128x128x80, 128 views, 37x37 PSF).

The CUDA path runs the full 128-view plan, in the launch configuration the
benchmark times; the oracle computes a sample of views exactly (each view of
A x depends on its own angle only, and A' of a projection set that is zero
outside the sampled views equals the oracle's A' over those views).  The EM
step is checked per step on a 4-view plan of the same volume and PSF, and at
128 views through properties that hold at any size.
"""
import numpy as np
import pytest

import oracle
from paper_2301_09710_gb300 import synthetic

from gpu_helpers import ADJ_FP32, PATHS, assert_close, dev, host, make_plan, need_gpu, oracle_psf, torch

pytestmark = pytest.mark.gpu

SAMPLE_VIEWS = [0, 17, 64, 101]


@pytest.fixture(scope="module")
def prob():
    need_gpu()
    return synthetic.config2(seed=0)


@pytest.mark.parametrize("path", PATHS)
def test_config2_sampled_views(prob, path):
    ang = oracle.default_angles(128)
    plan = make_plan(prob, ang, path)
    assert plan.info()["fused"] == (path in ("fused", "direct"))
    if plan.info()["fused"]:
        plan.autotune()  # the launch shapes the benchmark times
    x = dev(prob.x)
    v = host(plan.forward(x))
    psf = oracle_psf(prob, path)
    sub = ang[SAMPLE_VIEWS]
    v_o = oracle.forward(prob.x, prob.mu, psf, prob.dy, sub, nthreads=4)
    assert_close(v[SAMPLE_VIEWS], v_o, what="A x sampled views")
    # A' of a projection set supported on the sampled views
    rng = np.random.default_rng(5)
    y = np.zeros(plan.proj_shape, np.float32)
    y[SAMPLE_VIEWS] = rng.uniform(0, 1, (len(SAMPLE_VIEWS),) + plan.proj_shape[1:])
    xb = host(plan.back(dev(y)))
    xb_o = oracle.back(y[SAMPLE_VIEWS], prob.mu, psf, prob.dy, sub, nthreads=4)
    assert_close(xb, xb_o, what="A' y sampled views")
    plan.check()
    plan.close()


@pytest.mark.parametrize("path", ["fused", "lowmem"])
def test_config2_adjoint_and_em_invariants(prob, path):
    ang = oracle.default_angles(128)
    plan = make_plan(prob, ang, path)
    x = dev(prob.x)
    v = plan.forward(x)
    rng = np.random.default_rng(6)
    yy = rng.uniform(0, 1, plan.proj_shape).astype(np.float32)
    lhs = np.vdot(host(v), yy.astype(np.float64))
    rhs = np.vdot(prob.x.astype(np.float64), host(plan.back(dev(yy))))
    assert abs(lhs - rhs) <= ADJ_FP32 * abs(lhs)
    # EM with rbar = 0 keeps sum_j s_j x_j = sum_i y_i
    y = synthetic.poisson_counts(host(v) * (1e7 / host(v).sum()), 0)
    s = host(plan.sensitivity())
    xk = dev(np.where(prob.body, 1.0, 0.0).astype(np.float32))
    for _ in range(2):
        plan.em_step(xk, dev(y), None, niter=1)
        xs = host(xk)
        assert abs(np.sum(s * xs) - y.sum()) <= 1e-5 * y.sum()
        assert np.all(xs >= 0)
    # the fused EM step equals the composition of the library's own A and A'
    x0 = xk.clone()
    yb = plan.forward(x0)
    ratio = torch.where(yb > 0, dev(y) / yb, torch.zeros_like(yb))
    want = x0 * plan.back(ratio) / torch.from_numpy(s.astype(np.float32)).cuda()
    plan.em_step(xk, dev(y), None, niter=1)
    assert_close(host(xk), host(want), rel_l2=1e-6, max_rel=1e-5, what="fused EM vs composed")
    plan.check()
    plan.close()


@pytest.mark.parametrize("path", ["fused", "lowmem"])
def test_config2_geometry_em_step_vs_oracle(prob, path):
    views = [3, 40, 77, 120]
    ang = oracle.default_angles(128)[views]
    plan = make_plan(prob, ang, path)
    psf = oracle_psf(prob, path)
    xt = prob.x
    ybar = oracle.forward(xt, prob.mu, psf, prob.dy, ang, nthreads=4)
    scale = 1e7 / ybar.sum()
    y = synthetic.poisson_counts(ybar * scale, 1)
    rbar = synthetic.background_from((ybar * scale).astype(np.float32), 0.1, 8.0)
    x0 = np.where(prob.body, 1.0, 0.0).astype(np.float32)
    xg = dev(x0)
    plan.em_step(xg, dev(y), dev(rbar), niter=1)
    x1_o = oracle.em_step(x0, y, rbar, prob.mu, psf, prob.dy, ang, nthreads=4)
    assert_close(host(xg), x1_o, what="EM step, 128x128x80, 37x37 PSF")
    plan.close()


@pytest.mark.parametrize("shape", [(192, 128, 128, 37, [37]), (160, 96, 120, 29, [0, 53])],
                         ids=["192x192x128v128p37", "160x160x96v120p29"])
def test_large_planes_sampled_views(shape):
    """Planes too wide for one block's shared memory run on the column-tiled
    fused kernels (the serving workload's large case); sampled views against
    the oracle, adjointness over all views."""
    nx, nz, nview, p, views = shape
    x, mu, body = synthetic.small_phantom(nx, nz, 3)
    fx, fz = synthetic.depth_psf_factors(nx, p, p, 1.5, 9.0, aniso=True)
    prob = synthetic.Problem(x=x, mu=mu, dy=1.0, fx=fx, fz=fz, nview=nview, body=body, meta={})
    ang = oracle.default_angles(nview)
    plan = make_plan(prob, ang, "fused")
    assert plan.info()["fused"]
    psf = oracle_psf(prob, "fused")
    xg = dev(x)
    v = host(plan.forward(xg))
    assert_close(v[views], oracle.forward(x, mu, psf, 1.0, ang[views]), what="A x sampled views")
    rng = np.random.default_rng(8)
    y = np.zeros(plan.proj_shape, np.float32)
    y[views] = rng.uniform(0, 1, (len(views),) + plan.proj_shape[1:])
    assert_close(host(plan.back(dev(y))), oracle.back(y[views], mu, psf, 1.0, ang[views]), what="A' y sampled views")
    yy = rng.uniform(0, 1, plan.proj_shape).astype(np.float32)
    lhs = np.vdot(v, yy.astype(np.float64))
    rhs = np.vdot(x.astype(np.float64), host(plan.back(dev(yy))))
    assert abs(lhs - rhs) <= ADJ_FP32 * abs(lhs)
    plan.check()
    plan.close()


def test_benchmark_plan_all_views_vs_oracle(prob):
    """The benchmark's own problem and launch configuration, element by element:
    the 128-view plan autotuned as the benchmark tunes it, A x over all 128 views,
    A' y with y nonzero in every view (the view sum over all 128 views and the
    depth-group split of the autotuned shape), and one MLEM step with the smoothed
    10 % background, each against the FP64 oracle on all host threads."""
    from paper_2301_09710_gb300 import SpectPlan
    ang = oracle.default_angles(128)
    nz, ny, nx = prob.x.shape
    plan = SpectPlan(nx, nz, 128, mu=prob.mu, dy=prob.dy, fx=prob.fx, fz=prob.fz)
    plan.autotune()
    assert plan.info()["fused"]
    psf = oracle.psf_from_factors(prob.fx, prob.fz)
    v = host(plan.forward(dev(prob.x)))
    v_o = oracle.forward(prob.x, prob.mu, psf, prob.dy, ang)
    assert_close(v, v_o, what=f"A x, all 128 views, shape {plan.tuning}")
    rng = np.random.default_rng(11)
    y = rng.uniform(0.5, 1.5, plan.proj_shape).astype(np.float32)
    assert_close(host(plan.back(dev(y))), oracle.back(y, prob.mu, psf, prob.dy, ang),
                 what=f"A' y, all 128 views, shape {plan.tuning}")
    scale = 1e7 / v_o.sum()
    rbar = synthetic.background_from((v_o * scale).astype(np.float32), 0.1, 8.0)
    yc = synthetic.poisson_counts(v_o * scale + rbar, 0)
    x0 = np.where(prob.body, 1.0, 0.0).astype(np.float32)
    xg = dev(x0)
    plan.em_step(xg, dev(yc), dev(rbar), niter=1)
    assert_close(host(xg), oracle.em_step(x0, yc, rbar, prob.mu, psf, prob.dy, ang),
                 what="MLEM step, all 128 views")
    plan.check()
    plan.close()


# geometries whose planes do not fit one block's shared memory, so the fused
# kernels cut them into column tiles on their own (no tiling knob set)
LARGE = [(192, 128, 4, 37, 0.2), (256, 64, 4, 21, 0.1)]


@pytest.mark.parametrize("case", LARGE, ids=[f"{c[0]}x{c[1]}p{c[3]}" for c in LARGE])
def test_large_naturally_tiled_geometry_vs_oracle(case):
    from paper_2301_09710_gb300 import SpectPlan
    nx, nz, nv, p, mu_scale = case
    prob = synthetic.random_problem(nx + p, nx=nx, nz=nz, nview=nv, px=p, pz=p, mu_scale=mu_scale / nx * 16)
    ang = oracle.default_angles(nv) + 0.3
    plan = SpectPlan(nx, nz, nv, mu=prob.mu, dy=prob.dy, fx=prob.fx, fz=prob.fz, angles=ang)
    assert plan.info()["fused"] and plan.tuning["tiles"] > 1, plan.tuning
    psf = oracle.psf_from_factors(prob.fx, prob.fz)
    v = host(plan.forward(dev(prob.x)))
    assert_close(v, oracle.forward(prob.x, prob.mu, psf, prob.dy, ang), what=f"A x, {nx}x{nx}x{nz}, tiled")
    rng = np.random.default_rng(nx)
    y = rng.uniform(0.5, 2.0, v.shape)
    assert_close(host(plan.back(dev(y))), oracle.back(y, prob.mu, psf, prob.dy, ang),
                 what=f"A' y, {nx}x{nx}x{nz}, tiled")
    x0 = np.full(prob.x.shape, 0.5, np.float32)
    xg = dev(x0)
    plan.em_step(xg, dev(y), None, niter=1)
    assert_close(host(xg), oracle.em_step(x0, y, None, prob.mu, psf, prob.dy, ang),
                 what=f"EM step, {nx}x{nx}x{nz}, tiled")
    plan.check()
    plan.close()
