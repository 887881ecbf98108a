"""Three-pass rotation (Section II-A's alternative to bilinear rotation, reading
R13) on the fused kernels vs the FP64 oracle with rotation="3pass".

Same tolerances as the bilinear parity tests (relative L2 2e-6, per element
1e-4, FP32 adjoint mismatch 1e-5).  At quarter turns the two rotations are the
same lattice permutation, so the three-pass plan must give bitwise the
bilinear plan's results there.
"""
import numpy as np
import pytest

import oracle
from paper_2301_09710_gb300 import SpectPlan, synthetic

from gpu_helpers import ADJ_FP32, assert_close, dev, host, need_gpu, oracle_psf

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _plan(prob, ang, path, rotation="3pass"):
    nz, ny, nx = prob.x.shape
    if path == "fused":
        return SpectPlan(nx, nz, len(ang), mu=prob.mu, dy=prob.dy, fx=prob.fx, fz=prob.fz, angles=ang,
                         rotation=rotation)
    return SpectPlan(nx, nz, len(ang), mu=prob.mu, dy=prob.dy, psf=prob.full_psf(), angles=ang, rotation=rotation)


# (nx, nz, nview, psf size, seed, path): odd and even nx, nz not a multiple of 4
# or 32, several 16-column runs with a ragged one, separable and full PSFs
CASES = [(33, 12, 9, 5, 51, "fused"), (48, 20, 7, 9, 52, "fused"), (64, 16, 24, 37, 53, "fused"),
         (17, 5, 5, 3, 54, "fused"), (40, 8, 13, 11, 55, "direct"), (50, 36, 6, 7, 56, "fused")]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}v{c[2]}p{c[3]}{c[5]}" for c in CASES])
def test_rot3_forward_back_em_vs_oracle(case):
    nx, nz, nview, p, seed, path = case
    prob = synthetic.random_problem(seed, nx=nx, nz=nz, nview=nview, px=p, pz=p, mu_scale=0.1)
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, nview)
    psf = oracle_psf(prob, path)
    plan = _plan(prob, ang, path)
    assert plan.info()["fused"]
    x = dev(prob.x)
    v = host(plan.forward(x))
    assert_close(v, oracle.forward(prob.x, prob.mu, psf, prob.dy, ang, rotation="3pass"), what="A x (3-pass)")
    yy = rng.uniform(0, 1, plan.proj_shape).astype(np.float32)
    xb = host(plan.back(dev(yy)))
    assert_close(xb, oracle.back(yy, prob.mu, psf, prob.dy, ang, rotation="3pass"), what="A' y (3-pass)")
    lhs, rhs = np.vdot(v, yy.astype(np.float64)), np.vdot(prob.x.astype(np.float64), xb)
    assert abs(lhs - rhs) <= ADJ_FP32 * abs(lhs)
    # one EM step from the same FP32 iterate
    y = synthetic.poisson_counts(oracle.forward(prob.x, prob.mu, psf, prob.dy, ang, rotation="3pass") * 20, seed)
    x0 = np.full(prob.x.shape, 0.5, np.float32)
    xg = dev(x0)
    plan.em_step(xg, dev(y), None, niter=1)
    assert_close(host(xg), oracle.em_step(x0, y, None, prob.mu, psf, prob.dy, ang, rotation="3pass"),
                 what="EM step (3-pass)")
    # a different operator from the bilinear plan away from quarter turns
    bil = _plan(prob, ang, path, rotation="bilinear")
    vb = host(bil.forward(x))
    assert np.linalg.norm(v - vb) > 1e-4 * np.linalg.norm(v)
    plan.check()
    bil.check()


@pytest.mark.parametrize("path", ["fused", "direct"])
def test_rot3_quarter_turns_bitwise_equal_bilinear(path):
    prob = synthetic.random_problem(57, nx=24, nz=12, nview=8, px=7, pz=5, mu_scale=0.2)
    ang = np.arange(8) * np.pi / 2  # every view a quarter turn
    r3, bil = _plan(prob, ang, path), _plan(prob, ang, path, rotation="bilinear")
    x = dev(prob.x)
    assert np.array_equal(host(r3.forward(x)), host(bil.forward(x)))
    yy = dev(np.random.default_rng(57).uniform(0, 1, r3.proj_shape))
    np.testing.assert_allclose(host(r3.back(yy)), host(bil.back(yy)), rtol=1e-6, atol=1e-9)
    r3.check()
    bil.check()


def test_rot3_rejects_low_memory():
    from paper_2301_09710_gb300._lib import SpectError
    prob = synthetic.random_problem(58, nx=16, nz=4, nview=3, px=3, pz=3)
    with pytest.raises(SpectError, match="SPECT_EUNSUPPORTED"):
        SpectPlan(16, 4, 3, mu=prob.mu, dy=prob.dy, fx=prob.fx, fz=prob.fz, low_memory=True, rotation="3pass")


def test_rot3_config2_sampled_views():
    """The benchmark workload (128x128x80, 128 views, 37x37 separable PSF) with the
    three-pass rotation, autotuned; the oracle computes a sample of views."""
    prob = synthetic.config2(seed=0)
    ang = oracle.default_angles(128)
    plan = _plan(prob, ang, "fused")
    plan.autotune()
    views = [0, 17, 64, 101]
    psf = oracle_psf(prob, "fused")
    v = host(plan.forward(dev(prob.x)))
    assert_close(v[views], oracle.forward(prob.x, prob.mu, psf, prob.dy, ang[views], nthreads=4, rotation="3pass"),
                 what="A x sampled views (3-pass)")
    y = np.zeros(plan.proj_shape, np.float32)
    y[views] = np.random.default_rng(59).uniform(0, 1, (len(views),) + plan.proj_shape[1:])
    xb = host(plan.back(dev(y)))
    assert_close(xb, oracle.back(y[views], prob.mu, psf, prob.dy, ang[views], nthreads=4, rotation="3pass"),
                 what="A' y sampled views (3-pass)")
    plan.check()
    plan.close()


@pytest.mark.parametrize("case", [(33, 12, 9, 5, 61), (64, 16, 24, 37, 62)], ids=["33x12", "64x16"])
def test_rot3_patch_gather_bitwise_equals_list_gather(case, monkeypatch):
    """The patch gather stages boxes of the transposed pass-3 output and sums the
    four-entry lists in their order: A' and the EM update are bitwise those of the
    list gather."""
    nx, nz, nview, p, seed = case
    prob = synthetic.random_problem(seed, nx=nx, nz=nz, nview=nview, px=p, pz=p, mu_scale=0.1)
    ang = np.random.default_rng(seed).uniform(0, 2 * np.pi, nview)
    plan = _plan(prob, ang, "fused")
    monkeypatch.setenv("SPECT_GATHER", "0")
    ref = _plan(prob, ang, "fused")
    monkeypatch.delenv("SPECT_GATHER")
    assert plan.info()["device_bytes"] > ref.info()["device_bytes"]  # the patch boxes and entries
    yy = dev(np.random.default_rng(seed).uniform(0, 1, plan.proj_shape))
    assert np.array_equal(host(plan.back(yy)), host(ref.back(yy)))
    y = synthetic.poisson_counts(oracle.forward(prob.x, prob.mu, oracle_psf(prob, "fused"), prob.dy, ang,
                                                rotation="3pass") * 20, seed)
    x0 = np.full(prob.x.shape, 0.5, np.float32)
    xa, xr = dev(x0), dev(x0)
    plan.em_step(xa, dev(y), None, niter=2)
    ref.em_step(xr, dev(y), None, niter=2)
    assert np.array_equal(host(xa), host(xr))
    plan.check()
    ref.check()


@pytest.mark.parametrize("case", [(48, 20, 6, 11, 9, 1, 63, 3), (37, 13, 9, 5, 9, 9, 64, 2)],
                         ids=["48x20t3", "37x13t2vpsf"])
def test_rot3_column_tiled_and_view_dependent_psf(case, monkeypatch):
    """Column-tiled planes (the eight-tap rotation kernel's tile-image output) and
    a view-dependent PSF: parity with the oracle, and tiled A x bitwise equal to
    untiled."""
    nx, nz, nview, px, pz, nvp, seed, tiles = case
    prob = synthetic.random_problem(seed, nx=nx, nz=nz, nview=nview, px=px, pz=pz, nview_psf=nvp, mu_scale=0.1)
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, nview)
    psf = oracle_psf(prob, "fused")
    untiled = _plan(prob, ang, "fused")
    monkeypatch.setenv("SPECT_FUSED_TILES", str(tiles))
    plan = _plan(prob, ang, "fused")
    monkeypatch.delenv("SPECT_FUSED_TILES")
    assert plan.tuning["tiles"] > 1
    x = dev(prob.x)
    v = host(plan.forward(x))
    assert_close(v, oracle.forward(prob.x, prob.mu, psf, prob.dy, ang, rotation="3pass"), what="A x (3-pass, tiled)")
    assert np.array_equal(v, host(untiled.forward(x)))
    yy = rng.uniform(0, 1, plan.proj_shape).astype(np.float32)
    xb = host(plan.back(dev(yy)))
    assert_close(xb, oracle.back(yy, prob.mu, psf, prob.dy, ang, rotation="3pass"), what="A' y (3-pass, tiled)")
    assert np.array_equal(xb, host(untiled.back(dev(yy))))
    plan.check()
    untiled.check()
