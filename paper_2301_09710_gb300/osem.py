"""Ordered-subsets EM (OSEM): the EM update of Eqs. (7)-(8) (beta = 0) applied in
turn to M ordered subsets of the views, each with its own projector A_S and
sensitivity A_S'1 -- the reconstruction the paper runs with 4 subsets and 16
iterations when it compares projectors (Section III-A).

Subset m holds the views l = m (mod M), interleaved over the orbit.  Each
subset is a plan of the library over its views (angles and, for a
view-dependent PSF, its PSF rows), so a sub-iteration is one library EM step;
the data are split into subsets once, on the device.
"""
from __future__ import annotations

import numpy as np
import torch

from .projector import SpectPlan


def subsets(nview: int, n_subsets: int) -> list:
    """View indices of each ordered subset (interleaved)."""
    if not 1 <= n_subsets <= nview:
        raise ValueError("need 1 <= n_subsets <= nview")
    return [np.arange(m, nview, n_subsets) for m in range(n_subsets)]


class OSEM:
    """M plans over one geometry; `step` runs OSEM iterations in place."""

    def __init__(self, nx: int, nz: int, nview: int, n_subsets: int, mu=None, dy: float = 1.0, psf=None, fx=None,
                 fz=None, angles=None, device=None, **plan_kwargs):
        self.device = torch.device(device if device is not None else "cuda")
        self.nview, self.n_subsets = int(nview), int(n_subsets)
        ang = np.asarray(angles, dtype=np.float64) if angles is not None else \
            2.0 * np.pi * np.arange(nview, dtype=np.float64) / nview
        self.index = subsets(self.nview, self.n_subsets)

        def rows(a, idx):
            if a is None:
                return None
            a = np.asarray(a.cpu() if isinstance(a, torch.Tensor) else a)
            return a if a.shape[0] == 1 else np.ascontiguousarray(a[idx])

        self.plans = [SpectPlan(nx, nz, len(idx), mu=mu, dy=dy, psf=rows(psf, idx), fx=rows(fx, idx),
                                fz=rows(fz, idx), angles=ang[idx], device=self.device, **plan_kwargs)
                      for idx in self.index]
        self._dev_index = [torch.as_tensor(idx, device=self.device) for idx in self.index]

    def split(self, v):
        """Per-subset copies of projection data v (nview, nz, nx), or None."""
        if v is None:
            return [None] * self.n_subsets
        return [v.index_select(0, ix).contiguous() for ix in self._dev_index]

    def step(self, x, y_sub, rbar_sub=None, niter: int = 1, stream=None):
        """niter OSEM iterations of x in place; y_sub / rbar_sub from `split`."""
        rbar_sub = rbar_sub if rbar_sub is not None else [None] * self.n_subsets
        for _ in range(int(niter)):
            for plan, y, r in zip(self.plans, y_sub, rbar_sub):
                plan.em_step(x, y, r, niter=1, stream=stream)
        return x

    def check(self):
        for p in self.plans:
            p.check()

    def close(self):
        for p in self.plans:
            p.close()


def main(argv=None):
    """Time OSEM at the paper's setting (128x128x80, 128 views, 37x37 PSF, 4 subsets,
    16 iterations) against 16 MLEM iterations; print one JSON line."""
    import argparse
    import json

    ap = argparse.ArgumentParser(description="OSEM reconstruction timing")
    ap.add_argument("--subsets", type=int, default=4)
    ap.add_argument("--iters", type=int, default=16)
    a = ap.parse_args(argv)
    print(json.dumps(run(a.subsets, a.iters)))


def run(subsets: int = 4, iters: int = 16) -> dict:
    """OSEM (subsets x iters) against `iters` MLEM iterations on the paper-scale
    workload, timed with CUDA events after a warm-up run."""
    import argparse

    from . import synthetic
    a = argparse.Namespace(subsets=subsets, iters=iters)
    prob = synthetic.config2(seed=0)
    full = SpectPlan(128, 80, 128, mu=prob.mu, dy=prob.dy, fx=prob.fx, fz=prob.fz)
    xt = torch.from_numpy(prob.x).cuda()
    with torch.no_grad():
        primary = full.forward(xt)
        primary *= 1e7 / float(primary.sum())
    rbar_h = synthetic.background_from(primary.cpu().numpy(), 0.1, 8.0)
    y = torch.from_numpy(synthetic.poisson_counts(primary.cpu().numpy() + rbar_h, 0)).cuda()
    rbar = torch.from_numpy(rbar_h).cuda()
    x0 = torch.from_numpy(np.where(prob.body, 1.0, 0.0).astype(np.float32)).cuda()
    os_ = OSEM(128, 80, 128, a.subsets, mu=prob.mu, dy=prob.dy, fx=prob.fx, fz=prob.fz)
    ys, rs = os_.split(y), os_.split(rbar)
    out = {"workload": f"128x128x80, 128 views, 37x37 PSF, {a.subsets} subsets x {a.iters} iterations"}
    for name, run in (("osem", lambda x: os_.step(x, ys, rs, niter=a.iters)),
                      ("mlem", lambda x: full.em_step(x, y, rbar, niter=a.iters))):
        x = x0.clone()
        run(x)  # warm-up (sensitivities)
        x = x0.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run(x)
        e1.record()
        e1.synchronize()
        err = float(torch.linalg.norm(x - xt * (x.sum() / xt.sum())) / torch.linalg.norm(xt * (x.sum() / xt.sum())))
        out[name] = {"s": e0.elapsed_time(e1) / 1e3, "nrmsd_to_phantom": err}
    os_.check()
    full.check()
    os_.close()
    full.close()
    return out


if __name__ == "__main__":
    main()
