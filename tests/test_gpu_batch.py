"""Batches of plans run as one CUDA graph, and the launch-shape autotuner.

* every plan's EM iterates from the batch are bitwise those of the plan run
  alone (the graph replays the same kernel sequence on its own branch), on the
  first (captured) and a later (replayed) launch, and match the oracle;
* every launch shape the tuner may pick gives A, A' and EM within the FP32
  tolerance of the oracle, A' bitwise independent of the shape.
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


# nx, nz, nview, psf, seed, path -- uneven sizes, view counts and PSF widths
MIX = [(24, 8, 12, 5, 1, "fused"), (33, 12, 16, 11, 2, "fused"), (40, 7, 9, 7, 3, "fused"),
       (28, 10, 20, 3, 4, "lowmem"), (48, 16, 14, 9, 5, "fused")]


def _problems():
    out = []
    for nx, nz, nv, p, seed, path in MIX:
        prob = synthetic.config1(seed=seed, nx=nx, nz=nz, nview=nv, psf_size=p)
        ang = oracle.default_angles(nv)
        psf = oracle_psf(prob, path)
        ybar = oracle.forward(prob.x, prob.mu, psf, prob.dy, ang)
        y = synthetic.poisson_counts(ybar * 20, seed)
        rbar = np.full_like(y, 0.1 * float(y.mean()) + 0.01)
        x0 = np.where(prob.body, 1.0, 0.0).astype(np.float32) + 0.05
        out.append((prob, ang, psf, y, rbar, x0, path))
    return out


def test_batch_equals_each_plan_alone_and_the_oracle():
    from paper_2301_09710_gb300 import SpectBatch
    probs = _problems()
    plans = [make_plan(pr, ang, path) for pr, ang, psf, y, rb, x0, path in probs]
    ys = [dev(y) for _, _, _, y, _, _, _ in probs]
    rbs = [dev(rb) for _, _, _, _, rb, _, _ in probs]
    batch = SpectBatch(plans)
    niter = 3
    xs = [dev(x0) for *_, x0, _ in probs]
    batch.em_step(xs, ys, rbs, niter=niter)          # captured
    first = [host(x) for x in xs]
    for x, (*_, x0, _) in zip(xs, probs):
        x.copy_(dev(x0))
    batch.em_step(xs, ys, rbs, niter=niter)          # replayed
    again = [host(x) for x in xs]
    info = batch.info()
    assert info["plans"] == len(plans) and info["kernels_per_launch"] > len(plans) * niter
    batch.close()
    for i, (pl, (pr, ang, psf, y, rb, x0, path)) in enumerate(zip(plans, probs)):
        xa = dev(x0)
        pl.em_step(xa, ys[i], rbs[i], niter=niter)
        alone = host(xa)
        assert np.array_equal(first[i], alone), f"plan {i}: batch differs from the plan alone"
        assert np.array_equal(again[i], alone), f"plan {i}: replayed graph differs"
        s = oracle.sensitivity(pr.mu, psf, pr.dy, ang)
        xo = x0.astype(np.float64)
        for _ in range(niter):
            xo = oracle.em_step(xo, y, rb, pr.mu, psf, pr.dy, ang, s=s)
        assert_close(alone, xo, rel_l2=1e-5, max_rel=1e-3, what=f"plan {i} EM iterates vs oracle")
        pl.check()
        pl.close()


@pytest.mark.parametrize("shape", [(4, 4, 1), (16, 8, 2), (8, 16, 3), (4, 16, 4)])
def test_every_launch_shape_matches_the_oracle(shape):
    J, aJ, tiles = shape
    prob = synthetic.config1(seed=9, nx=40, nz=12, nview=10, psf_size=9)
    ang = oracle.default_angles(10)
    psf = oracle_psf(prob, "fused")
    ref = make_plan(prob, ang, "fused")
    plan = make_plan(prob, ang, "fused")
    plan.set_tuning(J, aJ, tiles)
    t = plan.tuning
    assert (t["fused_J"], t["adj_J"]) == (J, aJ) and t["tiles"] >= 1
    x = dev(prob.x)
    assert_close(host(plan.forward(x)), oracle.forward(prob.x, prob.mu, psf, prob.dy, ang), what="A x")
    rng = np.random.default_rng(3)
    yy = dev(rng.uniform(0, 1, plan.proj_shape))
    xb = host(plan.back(yy))
    assert_close(xb, oracle.back(host(yy), prob.mu, psf, prob.dy, ang), what="A' y")
    assert np.array_equal(xb, host(ref.back(yy))), "A' depends on the launch shape"
    y = synthetic.poisson_counts(oracle.forward(prob.x, prob.mu, psf, prob.dy, ang) * 10, 1)
    x0 = np.full(prob.x.shape, 0.7, np.float32)
    xg = dev(x0)
    plan.em_step(xg, dev(y), None, niter=1)
    assert_close(host(xg), oracle.em_step(x0, y, None, prob.mu, psf, prob.dy, ang), what="EM step")
    plan.check()


def test_autotune_picks_a_valid_shape_and_caches_it():
    prob = synthetic.config1(seed=4, nx=64, nz=32, nview=24, psf_size=11)
    ang = oracle.default_angles(24)
    psf = oracle_psf(prob, "fused")
    p1 = make_plan(prob, ang, "fused")
    t1 = p1.autotune()
    assert t1["fused_J"] in (4, 8, 12, 16, 20, 24, 32) and t1["adj_J"] in (4, 8, 12, 16, 20, 24, 32)
    assert t1["tiles"] >= 1
    p2 = make_plan(prob, ang, "fused")
    assert p2.autotune() == t1     # same geometry: the cached choice
    x = dev(prob.x)
    assert_close(host(p2.forward(x)), oracle.forward(prob.x, prob.mu, psf, prob.dy, ang), what="A x after tuning")
    p1.check()
    p2.check()
    # a low-memory plan has nothing to tune
    p3 = make_plan(prob, ang, "lowmem")
    p3.autotune()


# every plan on the fused separable kernels: the batch runs as grouped launches
FUSED_MIX = [(24, 8, 12, 5, 11), (33, 12, 16, 11, 12), (40, 8, 9, 7, 13), (48, 16, 14, 21, 14), (56, 20, 10, 9, 15),
             (40, 12, 11, 5, 16)]


def _fused_batch_inputs():
    out = []
    for nx, nz, nv, p, seed in FUSED_MIX:
        prob = synthetic.config1(seed=seed, nx=nx, nz=nz, nview=nv, psf_size=p)
        ang = oracle.default_angles(nv)
        psf = oracle_psf(prob, "fused")
        y = synthetic.poisson_counts(oracle.forward(prob.x, prob.mu, psf, prob.dy, ang) * 20, seed)
        rbar = np.full_like(y, 0.1 * float(y.mean()) + 0.01)
        x0 = np.where(prob.body, 1.0, 0.0).astype(np.float32) + 0.05
        out.append((prob, ang, psf, y, rbar, x0))
    return out


@pytest.mark.parametrize("branches", [1, 3])
def test_grouped_batch_equals_each_plan_alone(branches):
    """A batch whose plans all run the fused separable kernels runs each EM stage as
    one grouped launch over every plan (work items from all plans, the plans'
    arguments in the launch's parameters): fewer launches than a graph branch per
    plan, and every plan's iterates bitwise those of the plan alone and of the
    per-plan graph -- uneven sizes, view counts, five PSF buckets and a
    column-tiled plan."""
    from paper_2301_09710_gb300 import SpectBatch
    probs = _fused_batch_inputs()
    plans = [make_plan(pr, ang, "fused") for pr, ang, *_ in probs]
    t = plans[-1].tuning
    plans[-1].set_tuning(t["fused_J"], t["adj_J"], 2)  # column tiles: the tiled kernel variants
    assert plans[-1].tuning["tiles"] > 1
    ys = [dev(y) for _, _, _, y, _, _ in probs]
    rbs = [dev(rb) for _, _, _, _, rb, _ in probs]
    niter = 3
    runs = {}
    for mode in ("1", "0"):
        batch = SpectBatch(plans, grouped=branches if mode == "1" else 0)
        xs = [dev(x0) for *_, x0 in probs]
        batch.em_step(xs, ys, rbs, niter=niter)
        first = [host(x) for x in xs]
        for x, (*_, x0) in zip(xs, probs):
            x.copy_(dev(x0))
        batch.em_step(xs, ys, rbs, niter=niter)  # replayed
        runs[mode] = (first, [host(x) for x in xs], batch.info()["kernels_per_launch"])
        batch.close()
    assert runs["1"][2] < runs["0"][2], (runs["1"][2], runs["0"][2])
    for i, (pl, (pr, ang, psf, y, rb, x0)) in enumerate(zip(plans, probs)):
        xa = dev(x0)
        pl.em_step(xa, ys[i], rbs[i], niter=niter)
        alone = host(xa)
        for mode in ("1", "0"):
            assert np.array_equal(runs[mode][0][i], alone), f"plan {i}, grouped={mode}: differs from the plan alone"
            assert np.array_equal(runs[mode][1][i], alone), f"plan {i}, grouped={mode}: replay differs"
        if i < 2:
            s = oracle.sensitivity(pr.mu, psf, pr.dy, ang)
            xo = x0.astype(np.float64)
            for _ in range(niter):
                xo = oracle.em_step(xo, y, rb, pr.mu, psf, pr.dy, ang, s=s)
            assert_close(alone, xo, rel_l2=1e-5, max_rel=1e-3, what=f"plan {i} EM iterates vs oracle")
        pl.check()
        pl.close()
