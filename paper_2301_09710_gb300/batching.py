"""Batched EM reconstructions: many plans of uneven size, view count and PSF
width, their EM iterations captured as one CUDA graph (one branch per plan),
launch shapes picked by the library's autotuner.

``python -m paper_2301_09710_gb300.batching`` builds the workload (24
reconstructions with nx = ny in {64, 96, 128, 160}, nz in {32, 48, 64, 80, 96},
views in {60, 90, 120, 128}, PSF in {11, 21, 29, 37}, depth-dependent
Gaussians, ellipsoid phantoms, 8 EM iterations each) and times it three ways
with CUDA events: plan by plan on one stream (default launch shapes), as one
graph launch with default shapes, and as one graph launch after autotuning.
It prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def make_workload(n: int = 24, seed: int = 0, sizes=(64, 96, 128, 160), nzs=(32, 48, 64, 80, 96),
                  views=(60, 90, 120, 128), psfs=(11, 21, 29, 37)):
    """Seeded geometry, phantom, attenuation and PSF of every reconstruction."""
    from . import synthetic
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n):
        nx, nz, nv, p = (int(rng.choice(sizes)), int(rng.choice(nzs)), int(rng.choice(views)),
                         int(rng.choice(psfs)))
        x, mu, body = synthetic.small_phantom(nx, nz, seed * 1009 + r)
        fx, fz = synthetic.depth_psf_factors(nx, p, p, 1.0, 4.0, aniso=False)
        out.append(dict(nx=nx, nz=nz, nview=nv, psf=p, x=x, mu=mu, body=body, fx=fx, fz=fz))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="batched EM reconstructions as one CUDA graph")
    ap.add_argument("--plans", type=int, default=24)
    ap.add_argument("--niter", type=int, default=8)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    print(json.dumps(run(a.plans, a.niter, a.reps, a.seed)))


def run(n_plans: int = 24, niter: int = 8, reps: int = 3, seed: int = 0) -> dict:
    """Time the batching workload plan by plan and as one graph launch (default
    and autotuned launch shapes); returns the figures as a dict."""
    import torch

    from .projector import SpectBatch, SpectPlan
    a = argparse.Namespace(plans=n_plans, niter=niter, reps=reps, seed=seed)
    work = make_workload(a.plans, a.seed)
    dev = torch.device("cuda")
    st = torch.cuda.current_stream()
    t0 = time.perf_counter()
    plans, x0s, ys, rbs = [], [], [], []
    for w in work:
        pl = SpectPlan(w["nx"], w["nz"], w["nview"], mu=w["mu"], fx=w["fx"], fz=w["fz"], device=dev)
        xt = torch.from_numpy(w["x"]).to(dev)
        ybar = pl.forward(xt)
        rb = 0.1 * ybar.mean() * torch.ones_like(ybar)
        y = torch.poisson(ybar * 10 + rb)
        x0 = torch.from_numpy(np.where(w["body"], 1.0, 0.05).astype(np.float32)).to(dev)
        plans.append(pl)
        x0s.append(x0)
        ys.append(y)
        rbs.append(rb)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    xs = [x.clone() for x in x0s]

    def reset():
        for x, x0 in zip(xs, x0s):
            x.copy_(x0)

    def timed(fn):
        best = []
        for _ in range(a.reps):
            reset()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            e1.synchronize()
            best.append(e0.elapsed_time(e1) / 1e3)
        return float(np.median(best))

    def plain():
        for pl, x, y, rb in zip(plans, xs, ys, rbs):
            pl.em_step(x, y, rb, niter=a.niter)

    plain()  # warm-up (sensitivities)
    t_plain = timed(plain)
    ref = [x.clone() for x in xs]
    batch = SpectBatch(plans)
    batch.em_step(xs, ys, rbs, niter=a.niter)  # capture
    t_graph = timed(lambda: batch.em_step(xs, ys, rbs, niter=a.niter))
    same = all(torch.equal(x, r) for x, r in zip(xs, ref))
    kernels = batch.info()["kernels_per_launch"]
    batch.close()
    # the same batch as grouped launches (one per stage and kernel variant over the
    # blocks of every plan, in 1 and 4 branches), after the per-plan graph so its
    # one-pass slabs do not change the plan-by-plan runs above
    grouped = {}
    for nbr in (1, 4):
        batch = SpectBatch(plans, grouped=nbr)
        batch.em_step(xs, ys, rbs, niter=a.niter)
        tg = timed(lambda: batch.em_step(xs, ys, rbs, niter=a.niter))
        grouped[nbr] = {"recon_per_s": len(plans) / tg, "s": tg,
                        "kernels_per_graph_launch": batch.info()["kernels_per_launch"]}
        batch.close()
    t1 = time.perf_counter()
    tunings = [pl.autotune() for pl in plans]
    tune_s = time.perf_counter() - t1
    t_plain_tuned = timed(plain)
    batch = SpectBatch(plans)
    batch.em_step(xs, ys, rbs, niter=a.niter)
    t_graph_tuned = timed(lambda: batch.em_step(xs, ys, rbs, niter=a.niter))
    batch.close()
    for pl in plans:
        pl.check()
    n = len(plans)
    for pl in plans:
        pl.close()
    return ({
        "workload": f"{n} EM reconstructions x {a.niter} iterations, nx in {{64..160}}, nz in {{32..96}}, "
                    f"60-128 views, PSF 11-37 (separable depth-dependent Gaussians)",
        "geometries": [[w["nx"], w["nz"], w["nview"], w["psf"]] for w in work],
        "plain_s": t_plain, "graph_s": t_graph, "plain_tuned_s": t_plain_tuned, "graph_tuned_s": t_graph_tuned,
        "recon_per_s": {"plain": n / t_plain, "graph": n / t_graph, "graph_tuned": n / t_graph_tuned},
        "speedup_graph_tuned_vs_plain": t_plain / t_graph_tuned,
        "graph_bitwise_equal_to_plain": bool(same), "kernels_per_graph_launch": kernels,
        "grouped": {f"branches_{k}": v for k, v in grouped.items()},
        "setup_s": setup_s, "autotune_s": tune_s, "tunings": tunings,
    })


if __name__ == "__main__":
    main()
