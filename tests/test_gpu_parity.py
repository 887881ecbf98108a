"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (written here, derived in the design notes): relative L2 2e-6 and
per-element relative 1e-4 (denominator max(|o|, 1e-3 max|o|)) for A, A' and
one EM step from the same FP32 iterate; FP32 adjoint mismatch 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_2301_09710_gb300 import synthetic

from gpu_helpers import (ADJ_FP32, PATHS, assert_close, dev, host, make_plan, need_gpu, oracle_psf, torch)

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


# ---------------------------------------------------------------- config-1 workload, full size
@pytest.mark.parametrize("path", PATHS)
def test_config1_forward_back_em(path):
    prob = synthetic.config1(seed=0)
    ang = oracle.default_angles(prob.nview)
    psf = oracle_psf(prob, path)
    plan = make_plan(prob, ang, path)
    assert plan.info()["separable"] == (path in ("fused", "lowmem"))
    assert plan.info()["fused"] == (path in ("fused", "direct"))
    x = dev(prob.x)
    v = plan.forward(x)
    v_o = oracle.forward(prob.x, prob.mu, psf, prob.dy, ang)
    assert_close(host(v), v_o, what="A x")
    xb = plan.back(v)
    xb_o = oracle.back(v_o.astype(np.float32), prob.mu, psf, prob.dy, ang)
    assert_close(host(xb), xb_o, what="A' v")
    # one EM step from the same FP32 iterate
    y = synthetic.poisson_counts(v_o, 0)
    rbar = (0.1 * v_o.mean() * np.ones_like(v_o)).astype(np.float32)
    x0 = np.where(prob.body, 1.0, 0.0).astype(np.float32) + 0.05
    xg = dev(x0)
    plan.em_step(xg, dev(y), dev(rbar), niter=1)
    x1_o = oracle.em_step(x0, y, rbar, prob.mu, psf, prob.dy, ang)
    assert_close(host(xg), x1_o, what="EM step")
    # FP32 adjointness through the library
    rng = np.random.default_rng(1)
    yy = rng.uniform(0, 1, plan.proj_shape).astype(np.float32)
    lhs = np.vdot(host(plan.forward(x)), yy.astype(np.float64))
    rhs = np.vdot(prob.x.astype(np.float64), host(plan.back(dev(yy))))
    assert abs(lhs - rhs) <= ADJ_FP32 * abs(lhs)
    plan.check()
    plan.close()


# ---------------------------------------------------------------- ragged and degenerate shapes
CASES = [
    # nx, nz, nview, px, pz, nview_psf, seed
    (37, 13, 9, 5, 9, 9, 1),     # odd, ragged tiles, view-dependent PSF, pz wider than half nz
    (33, 1, 4, 7, 3, 1, 2),      # nz = 1: both k-edges fold on one row
    (2, 3, 3, 3, 5, 1, 3),       # smallest image
    (20, 40, 1, 1, 1, 1, 4),     # delta PSF, one view
    (48, 35, 7, 15, 11, 7, 5),   # PSF wider than tiles' halo multiple
]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}v{c[2]}p{c[3]}x{c[4]}" for c in CASES])
def test_ragged_forward_back(case, path):
    nx, nz, nview, px, pz, nvp, seed = case
    prob = synthetic.random_problem(seed, nx=nx, nz=nz, nview=nview, px=px, pz=pz, nview_psf=nvp, mu_scale=0.1)
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, nview)
    ang[0] = np.pi / 2  # always include an exact quarter turn
    psf = oracle_psf(prob, path)
    plan = make_plan(prob, ang, path)
    v = plan.forward(dev(prob.x))
    v_o = oracle.forward(prob.x, prob.mu, psf, prob.dy, ang)
    assert_close(host(v), v_o, what="A x")
    yy = rng.uniform(0, 1, plan.proj_shape).astype(np.float32)
    xb = plan.back(dev(yy))
    xb_o = oracle.back(yy, prob.mu, psf, prob.dy, ang)
    assert_close(host(xb), xb_o, what="A' y")
    plan.check()
    plan.close()


@pytest.mark.parametrize("low_memory", [False, True])
def test_no_attenuation_map(low_memory):
    prob = synthetic.random_problem(6, nx=24, nz=8, nview=5, px=5, pz=5)
    ang = oracle.default_angles(5)
    from paper_2301_09710_gb300 import SpectPlan
    plan = SpectPlan(24, 8, 5, mu=None, dy=1.0, fx=prob.fx, fz=prob.fz, angles=ang, low_memory=low_memory)
    v = plan.forward(dev(prob.x))
    v_o = oracle.forward(prob.x, np.zeros_like(prob.x), oracle.psf_from_factors(prob.fx, prob.fz), 1.0, ang)
    assert_close(host(v), v_o, what="A x, mu = 0")


@pytest.mark.parametrize("path", ["fused", "lowmem", "rot3"])
def test_strong_attenuation_over_many_depths(path):
    """Eq. (1) scanned over 100 depths (three full tiles of 32 and a ragged one)
    with attenuation up to about exp(-10) across the volume: A, A' and one EM
    step against the oracle."""
    from paper_2301_09710_gb300 import SpectPlan
    nx, nz, nv = 100, 8, 6
    prob = synthetic.random_problem(11, nx=nx, nz=nz, nview=nv, px=7, pz=5, mu_scale=0.2)
    ang = oracle.default_angles(nv)
    rot = "3pass" if path == "rot3" else "bilinear"
    plan = SpectPlan(nx, nz, nv, mu=prob.mu, dy=prob.dy, fx=prob.fx, fz=prob.fz, angles=ang,
                     low_memory=(path == "lowmem"), rotation=rot)
    psf = oracle.psf_from_factors(prob.fx, prob.fz)
    v = host(plan.forward(dev(prob.x)))
    assert_close(v, oracle.forward(prob.x, prob.mu, psf, prob.dy, ang, rotation=rot), what="A x, strong attenuation")
    rng = np.random.default_rng(12)
    y = rng.uniform(0.5, 2.0, v.shape)
    assert_close(host(plan.back(dev(y))), oracle.back(y, prob.mu, psf, prob.dy, ang, rotation=rot),
                 what="A' y, strong attenuation")
    x0 = np.full(prob.x.shape, 0.5, np.float32)
    xg = dev(x0)
    plan.em_step(xg, dev(y), None, niter=1)
    assert_close(host(xg), oracle.em_step(x0, y, None, prob.mu, psf, prob.dy, ang, rotation=rot),
                 what="EM step, strong attenuation")
    plan.check()
    plan.close()


@pytest.mark.parametrize("low_memory", [False, True])
def test_quarter_turns_exact_line_sums(low_memory):
    # mu = 0, delta PSF, views at multiples of 90 degrees: rotated line sums
    n, nz = 16, 5
    rng = np.random.default_rng(7)
    x = rng.integers(0, 8, (nz, n, n)).astype(np.float32)  # small integers: sums are exact in FP32
    from paper_2301_09710_gb300 import SpectPlan
    fx = np.zeros((1, n, 1), np.float32) + 1
    plan = SpectPlan(n, nz, 4, mu=None, dy=1.0, fx=fx, fz=fx.copy(), angles=np.arange(4) * np.pi / 2,
                     low_memory=low_memory)
    v = host(plan.forward(dev(x)))
    for q in range(4):
        want = np.stack([np.rot90(x[k], -q).sum(axis=0) for k in range(nz)])
        np.testing.assert_array_equal(v[q], want)


# ---------------------------------------------------------------- the paper's adjoint experiment
@pytest.mark.parametrize("path", PATHS)
def test_dense_adjoint_paper_shape_fp32(path):
    prob = synthetic.random_problem(100, nx=8, nz=6, nview=7, px=3, pz=3, symmetric=True, mu_scale=0.3)
    ang = oracle.default_angles(7)
    plan = make_plan(prob, ang, path)
    N, M = 8 * 8 * 6, 8 * 6 * 7
    eye_n = torch.eye(N, device="cuda", dtype=torch.float32)
    eye_m = torch.eye(M, device="cuda", dtype=torch.float32)
    A = np.stack([host(plan.forward(eye_n[c].reshape(plan.vol_shape))).ravel() for c in range(N)], axis=1)
    B = np.stack([host(plan.back(eye_m[r].reshape(plan.proj_shape))).ravel() for r in range(M)], axis=1)
    assert A.shape == (336, 384)
    err = np.linalg.norm(A.T - B) / np.linalg.norm(A)
    assert err < 1e-6, err  # the paper's FP32 figure (Section III-A)
    # and the dense matrix itself against the oracle's
    psf = oracle_psf(prob, path)
    A_o = np.stack([oracle.forward(e.reshape(6, 8, 8), prob.mu, psf, 1.0, ang, nthreads=1).ravel()
                    for e in np.eye(N)], axis=1)
    assert np.linalg.norm(A - A_o) / np.linalg.norm(A_o) < 2e-6


# ---------------------------------------------------------------- determinism
@pytest.mark.parametrize("path", PATHS)
def test_bitwise_deterministic(path):
    prob = synthetic.config1(seed=2, nx=32, nz=16, nview=16)
    ang = oracle.default_angles(16)
    plan = make_plan(prob, ang, path)
    x = dev(prob.x)
    a = host(plan.forward(x))
    b = host(plan.forward(x))
    np.testing.assert_array_equal(a, b)
    c = host(plan.back(dev(a)))
    d = host(plan.back(dev(a)))
    np.testing.assert_array_equal(c, d)


@pytest.mark.parametrize("path", PATHS)
def test_sensitivity_matches_oracle(path):
    prob = synthetic.config1(seed=3, nx=32, nz=12, nview=10, psf_size=7)
    ang = oracle.default_angles(10)
    plan = make_plan(prob, ang, path)
    s = host(plan.sensitivity())
    s_o = oracle.sensitivity(prob.mu, oracle_psf(prob, path), prob.dy, ang)
    assert_close(s, s_o, what="A'1")


# ---------------------------------------------------------------- column-tiled fused kernels
# (nx, nz, nview, px, pz, nview_psf, seed, tiles): planes cut into column tiles,
# including tiles narrower than the PSF halo and a ragged last tile
TILED = [
    (48, 20, 6, 11, 9, 1, 7, 3),
    (37, 13, 9, 5, 9, 9, 8, 2),
    (50, 7, 5, 15, 15, 1, 9, 4),
    (64, 16, 4, 37, 37, 1, 10, 4),
    (33, 1, 4, 7, 3, 1, 11, 3),
]


@pytest.mark.parametrize("case", TILED, ids=[f"{c[0]}x{c[1]}p{c[3]}t{c[7]}" for c in TILED])
def test_column_tiled_fused_kernels(case, monkeypatch):
    nx, nz, nview, px, pz, nvp, seed, tiles = case
    prob = synthetic.random_problem(seed, nx=nx, nz=nz, nview=nview, px=px, pz=pz, nview_psf=nvp, mu_scale=0.1)
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, nview)
    psf = oracle_psf(prob, "fused")
    untiled = make_plan(prob, ang, "fused")
    monkeypatch.setenv("SPECT_FUSED_TILES", str(tiles))
    plan = make_plan(prob, ang, "fused")
    monkeypatch.delenv("SPECT_FUSED_TILES")
    assert plan.info()["fused"]
    x = dev(prob.x)
    v = host(plan.forward(x))
    assert_close(v, oracle.forward(prob.x, prob.mu, psf, prob.dy, ang), what="A x, tiled")
    # only the data movement differs: the sums run in the same order
    assert np.array_equal(v, host(untiled.forward(x))), "tiled and untiled A x differ"
    yy = rng.uniform(0, 1, plan.proj_shape).astype(np.float32)
    xb = host(plan.back(dev(yy)))
    assert_close(xb, oracle.back(yy, prob.mu, psf, prob.dy, ang), what="A' y, tiled")
    assert np.array_equal(xb, host(untiled.back(dev(yy)))), "tiled and untiled A' y differ"
    y = synthetic.poisson_counts(oracle.forward(prob.x, prob.mu, psf, prob.dy, ang) * 30, seed)
    x0 = np.full(prob.x.shape, 0.5, np.float32)
    xg = dev(x0)
    plan.em_step(xg, dev(y), None, niter=1)
    assert_close(host(xg), oracle.em_step(x0, y, None, prob.mu, psf, prob.dy, ang), what="EM step, tiled")
    plan.check()
    plan.close()
    untiled.close()


# ---------------------------------------------------------------- patch-staged adjoint gather
GATHER = [(48, 20, 7, 9, 21), (33, 12, 9, 5, 22), (64, 16, 24, 37, 23), (17, 4, 5, 3, 24), (40, 8, 13, 11, 25),
          (56, 52, 6, 7, 26)]  # the last: four runs of k per patch (16, 16, 16, 4), a 7 x 7 patch grid


@pytest.mark.parametrize("case", GATHER, ids=[f"{c[0]}x{c[1]}v{c[2]}p{c[3]}" for c in GATHER])
def test_patch_gather_bitwise_equals_list_gather(case, monkeypatch):
    """The patch-staged gather (TMA boxes of the t slab) sums the same terms in
    the same order as the list gather: A' and the EM update are bitwise equal."""
    nx, nz, nview, p, seed = case
    prob = synthetic.random_problem(seed, nx=nx, nz=nz, nview=nview, px=p, pz=p, mu_scale=0.1)
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, nview)
    psf = oracle_psf(prob, "fused")
    plan = make_plan(prob, ang, "fused")
    monkeypatch.setenv("SPECT_GATHER", "0")
    ref = make_plan(prob, ang, "fused")
    monkeypatch.delenv("SPECT_GATHER")
    # the patch gather's boxes and entries are part of the plan's memory
    assert plan.info()["device_bytes"] > ref.info()["device_bytes"]
    yy = dev(rng.uniform(0, 1, plan.proj_shape))
    xb = host(plan.back(yy))
    assert np.array_equal(xb, host(ref.back(yy))), "patch gather differs from the list gather"
    assert_close(xb, oracle.back(host(yy), prob.mu, psf, prob.dy, ang), what="A' y (patch gather)")
    y = synthetic.poisson_counts(oracle.forward(prob.x, prob.mu, psf, prob.dy, ang) * 20, seed)
    x0 = np.full(prob.x.shape, 0.5, np.float32)
    xa, xr = dev(x0), dev(x0)
    plan.em_step(xa, dev(y), None, niter=2)
    ref.em_step(xr, dev(y), None, niter=2)
    assert np.array_equal(host(xa), host(xr)), "EM through the patch gather differs"
    plan.check()
    ref.check()


# ---------------------------------------------------------------- patch-staged forward rotation
ROTP = [(48, 20, 7, 9, 31, "fused"), (33, 12, 9, 5, 32, "fused"), (64, 16, 24, 37, 33, "fused"),
        (17, 4, 5, 3, 34, "fused"), (40, 8, 13, 11, 35, "direct"), (50, 36, 6, 7, 36, "fused")]


@pytest.mark.parametrize("case", ROTP, ids=[f"{c[0]}x{c[1]}v{c[2]}p{c[3]}{c[5]}" for c in ROTP])
def test_patch_rotation_bitwise_equals_plane_rotation(case, monkeypatch):
    """The patch-staged rotation (x_t boxes and attenuation tiles by TMA) computes
    every sample with the same weights, corners and arithmetic as the plane
    gather: A x and the EM update are bitwise equal."""
    nx, nz, nview, p, seed, path = case
    prob = synthetic.random_problem(seed, nx=nx, nz=nz, nview=nview, px=p, pz=p, mu_scale=0.1)
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, nview)
    psf = oracle_psf(prob, path)
    monkeypatch.setenv("SPECT_ROTPATCH", "1")  # patch rotation from the start
    plan = make_plan(prob, ang, path)
    monkeypatch.setenv("SPECT_ROTPATCH", "0")
    ref = make_plan(prob, ang, path)
    monkeypatch.delenv("SPECT_ROTPATCH")
    assert plan.info()["device_bytes"] > ref.info()["device_bytes"]  # the patch boxes
    x = dev(prob.x)
    v = host(plan.forward(x))
    assert np.array_equal(v, host(ref.forward(x))), "patch rotation differs from the plane rotation"
    assert_close(v, oracle.forward(prob.x, prob.mu, psf, prob.dy, ang), what="A x (patch rotation)")
    y = synthetic.poisson_counts(oracle.forward(prob.x, prob.mu, psf, prob.dy, ang) * 20, seed)
    x0 = np.full(prob.x.shape, 0.5, np.float32)
    xa, xr = dev(x0), dev(x0)
    plan.em_step(xa, dev(y), None, niter=2)
    ref.em_step(xr, dev(y), None, niter=2)
    assert np.array_equal(host(xa), host(xr)), "EM through the patch rotation differs"
    plan.check()
    ref.check()


# ---------------------------------------------------------------- 16-iteration EM trajectory
def test_em_trajectory_drift_16_iterations():
    """The GPU's own FP32 iterates over 16 MLEM iterations against the FP64 oracle's
    (not re-synchronised per step): the drift grows about linearly in k and stays
    within the per-step bars (measured 4.8e-8 at k = 1 to 3.1e-7 at k = 16, rel L2)."""
    prob = synthetic.config1(seed=0)
    ang = oracle.default_angles(prob.nview)
    psf = oracle_psf(prob, "fused")
    plan = make_plan(prob, ang, "fused")
    v = oracle.forward(prob.x, prob.mu, psf, prob.dy, ang)
    y = synthetic.poisson_counts(v * (1e6 / v.sum()), 0)
    x0 = np.where(prob.body, 1.0, 0.0).astype(np.float32)
    xg, yg = dev(x0), dev(y)
    s = oracle.sensitivity(prob.mu, psf, prob.dy, ang)
    xo = x0.astype(np.float64)
    drift = []
    for _ in range(16):
        plan.em_step(xg, yg, None, niter=1)
        xo = oracle.em_step(xo, y, None, prob.mu, psf, prob.dy, ang, s=s)
        e2, emax = assert_close(host(xg), xo, what=f"EM iterate {len(drift) + 1} (trajectory)")
        drift.append(e2)
    assert drift[-1] < 16 * max(drift[0], 1e-8)  # no faster than linear growth
    plan.check()
