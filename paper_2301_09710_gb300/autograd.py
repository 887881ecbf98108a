"""Differentiation through the projector (Section II-A: the backward pass of A is A', written by hand)
and the unrolled CNN-regularised EM of Algorithm 3 (Section II-B).

* ``project(x, plan)`` is A x with backward A' g; ``backproject(v, plan)`` is A' v
  with backward A g.  Both run the library's kernels (the transpose is exact, so
  these are the true Jacobians) and never store rotated intermediates.
* ``em_update`` is one inner iteration of Eqs. (7)-(8) written with them and
  with the library's element-wise EM kernels (the ratio y / (A x + rbar) and the
  closed-form update, each with a hand-written gradient kernel: the implicit
  derivative of beta x+^2 + d x+ - x e = 0), so gradients flow through A, A' and
  the update with every step in the library's kernels.
* ``UnrolledEM`` unrolls K outer iterations u = g_theta(x_k), x_{k+1} = EM(x_k, u)
  with a small 3D CNN g_theta and per-iteration activation checkpointing
  (``torch.utils.checkpoint``): only the iterates are kept, everything inside an
  iteration is recomputed in the backward pass.

The CNN uses torch's conv3d (it is not part of the projector path).
"""
from __future__ import annotations

import torch
import torch.nn as nn
import torch.utils.checkpoint as ckpt

from . import projector as _pj
from .projector import SpectPlan


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return plan.forward(x.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.back(g.contiguous()), None


class _BackProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, plan):
        ctx.plan = plan
        return plan.back(v.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.forward(g.contiguous()), None


def project(x: torch.Tensor, plan) -> torch.Tensor:
    """v = A x, differentiable (backward: A')."""
    return _Project.apply(x, plan)


def backproject(v: torch.Tensor, plan) -> torch.Tensor:
    """x = A' v, differentiable (backward: A)."""
    return _BackProject.apply(v, plan)


class _Ratio(torch.autograd.Function):
    """y / (ybar + rbar) (0 where ybar + rbar <= 0); differentiable in ybar."""

    @staticmethod
    def forward(ctx, ybar, y, rbar):
        ybar, y = ybar.contiguous(), y.contiguous()
        rbar = rbar.contiguous() if rbar is not None else None
        ctx.save_for_backward(ybar, y, rbar)
        return _pj.em_ratio(ybar, y, rbar)

    @staticmethod
    def backward(ctx, g):
        ybar, y, rbar = ctx.saved_tensors
        return _pj.em_ratio_backward(ybar, y, rbar, g.contiguous()), None, None


class _Update(torch.autograd.Function):
    """The closed-form update of Eqs. (7)-(8); differentiable in x, e and u."""

    @staticmethod
    def forward(ctx, x, e, s, u, beta):
        x, e, s = x.contiguous(), e.contiguous(), s.contiguous()
        u = u.contiguous() if (u is not None and beta > 0) else None
        ctx.beta = float(beta)
        ctx.save_for_backward(x, e, s, u)
        return _pj.em_update(x, e, s, u, float(beta))

    @staticmethod
    def backward(ctx, g):
        x, e, s, u = ctx.saved_tensors
        gx, ge, gu = _pj.em_update_backward(x, e, s, u, ctx.beta, g.contiguous())
        return gx, ge, None, gu, None


def em_ratio(ybar, y, rbar):
    return _Ratio.apply(ybar, y, rbar)


def em_root(x, e, s, u, beta):
    return _Update.apply(x, e, s, u, beta)


def em_update(x, y, rbar, plan, s, u=None, beta: float = 0.0):
    """One inner EM iteration, Eqs. (7)-(8), differentiable in x and u.

    beta == 0: x e / s (MLEM).  beta > 0: the non-negative root of
    beta x'^2 + d x' - x e = 0, d = s - beta u, in the cancellation-free form
    for the sign of d.  Guards as the library: ratio 0 where A x + rbar <= 0,
    voxel 0 where the root is not finite and positive.  Every step runs in the
    library's kernels: A, the ratio, A', the update (and their gradients).
    """
    ratio = em_ratio(project(x, plan), y, rbar)
    e = backproject(ratio, plan)
    if beta == 0.0 or u is None:
        return em_root(x, e, s, None, 0.0)
    return em_root(x, e, s, u, beta)


class Regularizer3D(nn.Module):
    """g_theta: 3 conv3d layers (3x3x3), ReLU between them, residual on the input
    (Section III-B: a 3-layer CNN with ReLU except after the last layer)."""

    def __init__(self, channels: int = 8):
        super().__init__()
        self.c1 = nn.Conv3d(1, channels, 3, padding=1)
        self.c2 = nn.Conv3d(channels, channels, 3, padding=1)
        self.c3 = nn.Conv3d(channels, 1, 3, padding=1)
        for m in (self.c1, self.c2, self.c3):
            nn.init.normal_(m.weight, std=0.02)
            nn.init.zeros_(m.bias)

    def forward(self, x):  # x: (nz, ny, nx)
        h = x[None, None]
        h = torch.relu(self.c1(h))
        h = torch.relu(self.c2(h))
        return x + self.c3(h)[0, 0]


class UnrolledEM(nn.Module):
    """Algorithm 3 unrolled: K outer iterations of u = g(x_k) and n_inner EM updates.

    ``checkpoint=True`` recomputes each outer iteration in the backward pass, so
    memory holds only the K+1 iterates (the paper's motivation for end-to-end
    training without storing rotated intermediates, Section IV).
    """

    def __init__(self, plan: SpectPlan, n_outer: int = 3, n_inner: int = 1, beta: float = 1.0,
                 channels: int = 8, checkpoint: bool = True, cnn: nn.Module | None = None):
        super().__init__()
        self.plan = plan
        self.n_outer, self.n_inner, self.beta = int(n_outer), int(n_inner), float(beta)
        self.cnn = cnn if cnn is not None else Regularizer3D(channels)
        self.checkpoint = checkpoint
        self._s = None

    def sensitivity(self):
        if self._s is None:
            with torch.no_grad():
                self._s = self.plan.sensitivity()
        return self._s

    def outer(self, x, y, rbar):
        s = self.sensitivity()
        u = self.cnn(x)
        for _ in range(self.n_inner):
            x = em_update(x, y, rbar, self.plan, s, u, self.beta)
        return x

    def forward(self, x0, y, rbar=None):
        x = x0
        for _ in range(self.n_outer):
            if self.checkpoint and torch.is_grad_enabled():
                x = ckpt.checkpoint(self.outer, x, y, rbar, use_reentrant=False)
            else:
                x = self.outer(x, y, rbar)
        return x


def main(argv=None):
    """Time one training step of the unrolled network at the paper's scale
    (128x128x80, 128 views, 37x37 PSF, 8 outer iterations of a 3-layer 8-channel
    CNN + 1 EM update, MSE to the phantom), with and without checkpointing, and
    print one JSON line (ms per step, peak device memory)."""
    import argparse
    import json

    ap = argparse.ArgumentParser(description="unrolled CNN-regularised EM: one training step")
    ap.add_argument("--outer", type=int, default=8)
    ap.add_argument("--channels", type=int, default=8)
    ap.add_argument("--beta", type=float, default=1.0)
    ap.add_argument("--steps", type=int, default=3)
    a = ap.parse_args(argv)
    print(json.dumps(run(a.outer, a.channels, a.beta, a.steps)))


def run(outer: int = 8, channels: int = 8, beta: float = 1.0, steps: int = 3) -> dict:
    """One training step of the unrolled network at the paper's scale, timed with
    CUDA events (median of `steps`), with and without checkpointing."""
    import argparse

    import numpy as np

    from . import synthetic
    a = argparse.Namespace(outer=outer, channels=channels, beta=beta, steps=steps)
    dev = torch.device("cuda")
    prob = synthetic.config2(seed=0)
    plan = SpectPlan(128, 80, 128, mu=prob.mu, dy=prob.dy, fx=prob.fx, fz=prob.fz, device=dev)
    plan.autotune()
    xt = torch.from_numpy(prob.x).to(dev)
    with torch.no_grad():
        primary = plan.forward(xt)
        scale = 1e7 / float(primary.sum())
    target = xt * scale
    primary = (primary * scale).cpu().numpy()
    rbar = torch.from_numpy(synthetic.background_from(primary, 0.1, 8.0)).to(dev)
    y = torch.from_numpy(synthetic.poisson_counts(primary + rbar.cpu().numpy(), 0)).to(dev)
    x0 = torch.from_numpy(np.where(prob.body, 1.0, 0.0).astype(np.float32)).to(dev) * float(target.mean())
    out = {"workload": "unrolled EM, 128x128x80 image, 128 views, 37x37 PSF, "
                       f"{a.outer} outer iterations x (3-layer {a.channels}-channel 3D CNN + 1 EM update), MSE loss"}
    for ck in (True, False):
        torch.manual_seed(0)
        net = UnrolledEM(plan, n_outer=a.outer, n_inner=1, beta=a.beta, channels=a.channels, checkpoint=ck).to(dev)
        opt = torch.optim.Adam(net.cnn.parameters(), lr=1e-4)
        times = []
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        for it in range(a.steps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            opt.zero_grad(set_to_none=True)
            loss = ((net(x0, y, rbar) - target) ** 2).mean()
            loss.backward()
            opt.step()
            e1.record()
            e1.synchronize()
            if it > 0:
                times.append(e0.elapsed_time(e1))
        key = "checkpointed" if ck else "stored"
        out[key] = {"ms_per_step": float(np.median(times)), "loss": loss.item(),
                    "peak_device_gb": torch.cuda.max_memory_allocated() / 2**30}
    plan.check()
    plan.close()
    return out


if __name__ == "__main__":
    main()
