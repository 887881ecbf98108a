"""Continuous-batching EM reconstruction server.

Requests (an attenuation map, a PSF, angles, measured projections, a background
and an iteration count) arrive over time.  The server admits a request as soon
as its device memory fits the free budget and a slot is free, keeps its plan,
iterate, data and background resident on the GPU, and interleaves the MLEM
iterations (Eqs. (7)-(8), beta = 0) of all admitted requests round-robin over a
set of CUDA streams, so iterations of different requests run concurrently and
small reconstructions fill the SMs a single one leaves idle.  A finished
request's image is copied back, its plan released and its slot reused at once.

``serve_plain`` runs the same requests one at a time through the same library
calls (the baseline the server is compared with).

Admission is by free device memory: the budget is the device's free memory
when the server starts (``cudaMemGetInfo``, less a reserve), and before each
admission the device's live free memory is checked again, less what admitted
requests whose plans are still being built will take, so memory taken by
anything else on the device holds requests back.

The scheduler is host logic over an ``Executor``; ``GpuExecutor`` drives the
library, ``FakeExecutor`` (tests) simulates device memory and a kernel clock
without a GPU.
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds from the start of the run
    nx: int
    nz: int
    nview: int
    niter: int
    mu: np.ndarray                 # (nz, nx, nx) float32
    fx: np.ndarray                 # (1, nx, px)
    fz: np.ndarray                 # (1, nx, pz)
    y: np.ndarray                  # (nview, nz, nx)
    rbar: np.ndarray | None = None
    x0: np.ndarray | None = None
    dy: float = 1.0


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    done: float
    x: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


# --------------------------------------------------------------------------- executors
class GpuExecutor:
    """Runs requests on one GPU through the library (one plan per request).

    Plans are built on a host worker thread (the library call releases the
    interpreter lock), so the scheduler keeps feeding the other requests'
    streams meanwhile; plan memory is stream-ordered, and a finished request
    synchronises and releases only its own stream.  ``iters_per_step`` EM
    iterations are enqueued per scheduling turn.
    """

    def __init__(self, device="cuda", n_streams: int = 4, keep_images: bool = True, iters_per_step: int = 2):
        import concurrent.futures as cf
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_streams)]
        self.keep_images = keep_images
        self.iters_per_step = max(1, int(iters_per_step))
        self.pool = cf.ThreadPoolExecutor(max_workers=1)
        self.plan_bytes_seen = []
        self._pending = {}          # id(handle) -> bytes promised to a plan still being built
        self.t0 = time.perf_counter()

    def free_bytes(self) -> int:
        """Device memory free right now: cudaMemGetInfo's free bytes plus what
        torch's caching allocator holds unused (reusable by request tensors)."""
        torch = self.torch
        free, _total = torch.cuda.mem_get_info(self.device)
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        return int(free + max(0, cached))

    def pending_bytes(self) -> int:
        """Memory promised to admitted requests whose plans are not built yet
        (not visible in free_bytes() until they are)."""
        return int(sum(self._pending.values()))

    def now(self) -> float:
        return time.perf_counter() - self.t0

    @staticmethod
    def plan_bytes(req: Request, compact: bool = False) -> int:
        """Device memory one request holds while admitted: the library's bound
        on its plan (spect_plan_bytes), plus iterate, data and background, plus
        slack for allocator rounding.  compact: the plan recomputes the
        attenuation per view chunk (SPECT_PLAN_RECOMPUTE_ATTENUATION) instead
        of caching it for every view."""
        from .projector import plan_bytes
        nvp, _, px = req.fx.shape
        pz = req.fz.shape[-1]
        plan = plan_bytes(req.nx, req.nz, req.nview, px, pz, nvp, separable=True, recompute_attenuation=compact)
        tensors = 4 * (req.nx * req.nx * req.nz + 2 * req.nview * req.nz * req.nx)
        return int((plan + tensors) * 1.02) + (8 << 20)

    def _create(self, req: Request, st, compact: bool = False):
        from .projector import SpectPlan
        torch = self.torch
        with torch.cuda.device(self.device), torch.cuda.stream(st):
            plan = SpectPlan(req.nx, req.nz, req.nview, mu=req.mu, dy=req.dy, fx=req.fx, fz=req.fz,
                             device=self.device, stream=st, recompute_attenuation=compact)
            x0 = req.x0 if req.x0 is not None else np.ones((req.nz, req.nx, req.nx), np.float32)
            x = torch.from_numpy(np.ascontiguousarray(x0, np.float32)).to(self.device)
            y = torch.from_numpy(np.ascontiguousarray(req.y, np.float32)).to(self.device)
            rb = None
            if req.rbar is not None:
                rb = torch.from_numpy(np.ascontiguousarray(req.rbar, np.float32)).to(self.device)
        self.plan_bytes_seen.append((req.rid, plan.info()["device_bytes"]))
        return plan, x, y, rb

    def start(self, req: Request, slot: int, compact: bool = False):
        st = self.streams[slot % len(self.streams)]
        h = {"future": self.pool.submit(self._create, req, st, compact), "plan": None, "stream": st,
             "left": req.niter, "event": None}
        self._pending[id(h)] = self.plan_bytes(req, compact)
        return h

    def step(self, h) -> None:
        """Enqueue the next EM iterations of a request on its stream (asynchronous)."""
        torch = self.torch
        n = min(self.iters_per_step, h["left"])
        with torch.cuda.stream(h["stream"]):
            h["plan"].em_step(h["x"], h["y"], h["rbar"], niter=n, stream=h["stream"])
            ev = torch.cuda.Event()
            ev.record(h["stream"])
        h["event"] = ev
        h["left"] -= n

    def ready(self, h) -> bool:
        if h["plan"] is None:
            if not h["future"].done():
                return False
            h["plan"], h["x"], h["y"], h["rbar"] = h["future"].result()
            self._pending.pop(id(h), None)
        return h["event"] is None or h["event"].query()

    def finish(self, h):
        torch = self.torch
        plan, st = h["plan"], h["stream"]
        plan.check(stream=st)
        x = None
        if self.keep_images:
            with torch.cuda.stream(st):
                x = h["x"].cpu().numpy()
        plan.release(st)
        return x

    def close(self):
        self.pool.shutdown(wait=True)


class FakeExecutor:
    """Simulated device for scheduler tests: a memory figure per request and a
    clock; every admitted request's EM iteration takes ``iter_cost`` and
    iterations of different requests overlap fully.  ``device_bytes`` is the
    simulated device memory (None: unlimited); ``other_use(t)`` is memory taken
    at time t by something other than the server."""

    def __init__(self, iter_cost: float = 0.01, plan_cost: float = 0.0, device_bytes=None, other_use=None):
        self.t = 0.0
        self.iter_cost, self.plan_cost = iter_cost, plan_cost
        self.device_bytes = device_bytes
        self.other_use = other_use
        self.held = 0
        self.log = []

    def now(self) -> float:
        return self.t

    def free_bytes(self):
        if self.device_bytes is None:
            return None
        other = self.other_use(self.t) if self.other_use else 0
        return self.device_bytes - self.held - other

    @staticmethod
    def pending_bytes() -> int:
        return 0

    @staticmethod
    def plan_bytes(req: Request, compact: bool = False) -> int:
        full = req.nx * req.nx * req.nz * req.nview
        return full // 4 if compact else full  # a compact plan: a quarter of the memory

    def start(self, req, slot, compact: bool = False):
        self.t += self.plan_cost
        self.held += self.plan_bytes(req, compact)
        self.log.append(("start", req.rid, self.t, compact))
        return {"rid": req.rid, "left": req.niter, "busy_until": self.t, "bytes": self.plan_bytes(req, compact)}

    def step(self, h):
        h["busy_until"] = max(h["busy_until"], self.t) + self.iter_cost
        h["left"] -= 1

    def ready(self, h):
        return h["busy_until"] <= self.t + 1e-12

    def advance(self, active, next_arrival=None):
        """Move the clock to the next completion or arrival."""
        cands = [h["busy_until"] for h in active if h["busy_until"] > self.t]
        if next_arrival is not None and next_arrival > self.t:
            cands.append(next_arrival)
        if cands:
            self.t = min(cands)

    def finish(self, h):
        self.held -= h["bytes"]
        self.log.append(("finish", h["rid"], self.t))
        return None


# --------------------------------------------------------------------------- scheduler
@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    makespan: float = 0.0
    peak_bytes: int = 0
    peak_active: int = 0
    held_back: int = 0          # admissions deferred because the device's live free memory was short
    compact: int = 0            # requests admitted with a compact plan (compact_fallback)
    budget: int = 0

    def summary(self) -> dict:
        lat = np.array([r.latency for r in self.results]) if self.results else np.zeros(1)
        return {"requests": len(self.results), "recon_per_s": len(self.results) / max(self.makespan, 1e-9),
                "p50_s": float(np.percentile(lat, 50)), "p95_s": float(np.percentile(lat, 95)),
                "p99_s": float(np.percentile(lat, 99)), "makespan_s": self.makespan,
                "peak_active": self.peak_active, "peak_bytes": self.peak_bytes, "budget_bytes": self.budget,
                "held_back_by_free_memory": self.held_back, "compact_admissions": self.compact}


RESERVE_BYTES = 2 << 30  # device memory the server leaves free for everything else


def serve(requests, executor, mem_budget=None, max_active: int = 16, poll_sleep: float = 0.0,
          reserve_bytes: int = RESERVE_BYTES, compact_fallback: bool = False) -> ServeStats:
    """Continuous batching: admit by memory and slots, interleave EM iterations
    round-robin, retire finished requests immediately.

    mem_budget: bytes the server may hold at once; None takes the device's free
    memory at the start less ``reserve_bytes``.  Each admission also needs the
    request's bytes free on the device at that moment (live free memory, less
    the bytes of plans still being built, less the reserve), unless nothing is
    admitted (memory released in stream order may not show as free yet).

    compact_fallback: a request whose plan does not fit now is admitted with a
    compact plan (the attenuation recomputed per view chunk, a fraction of the
    memory, slower iterations) when that fits, instead of waiting.  Its image
    then matches the caching plan's within the FP32 tolerance rather than bit for
    bit (its back-projection sums the views in chunks)."""
    free0 = executor.free_bytes() if hasattr(executor, "free_bytes") else None
    if mem_budget is None:
        if free0 is None:
            raise ValueError("mem_budget is required when the executor cannot report free device memory")
        mem_budget = free0 - reserve_bytes
    pending = sorted(requests, key=lambda r: r.arrival)
    queue: list = []            # arrived, not admitted (FIFO)
    active: list = []           # (request, handle, admitted_at, slot)
    used = 0
    slots_free = list(range(max_active))
    stats = ServeStats()
    stats.budget = int(mem_budget)
    pi = 0

    def short_of(n):  # None if n more bytes fit now, else what they are short of
        if used + n > mem_budget:
            return "budget"
        if active and free0 is not None:
            live = executor.free_bytes() - executor.pending_bytes() - reserve_bytes
            if n > live:
                return "live"
        return None

    while pi < len(pending) or queue or active:
        now = executor.now()
        while pi < len(pending) and pending[pi].arrival <= now:
            queue.append(pending[pi])
            pi += 1
        # admission in arrival order while memory and slots allow
        while queue and slots_free:
            need, compact = executor.plan_bytes(queue[0]), False
            smallest = min(need, executor.plan_bytes(queue[0], compact=True)) if compact_fallback else need
            if smallest > mem_budget:
                raise ValueError(f"request {queue[0].rid} needs {smallest} bytes, more than the whole budget")
            short = short_of(need)
            if short and smallest < need and short_of(smallest) is None:
                need, compact, short = smallest, True, None
            if short:
                if short == "live":
                    stats.held_back += 1
                break
            req = queue.pop(0)
            slot = slots_free.pop(0)
            h = executor.start(req, slot, compact) if compact else executor.start(req, slot)
            stats.compact += int(compact)
            used += need
            active.append([req, h, executor.now(), slot, need])
            stats.peak_bytes = max(stats.peak_bytes, used)
        stats.peak_active = max(stats.peak_active, len(active))
        # one iteration for every admitted request whose previous one is done
        progressed = False
        for a in list(active):
            req, h = a[0], a[1]
            if not executor.ready(h):
                continue
            if h["left"] > 0:
                executor.step(h)
                progressed = True
            else:
                x = executor.finish(h)
                stats.results.append(Result(req.rid, req.arrival, a[2], executor.now(), x))
                active.remove(a)
                used -= a[4]
                slots_free.append(a[3])
                progressed = True
        if isinstance(executor, FakeExecutor):
            if not progressed:
                executor.advance([a[1] for a in active], pending[pi].arrival if pi < len(pending) else None)
        elif not progressed:
            if not active and pi < len(pending):
                time.sleep(max(0.0, min(pending[pi].arrival - executor.now(), 0.01)))
            elif poll_sleep:
                time.sleep(poll_sleep)
    stats.makespan = executor.now()
    stats.results.sort(key=lambda r: r.rid)
    return stats


def serve_plain(requests, executor) -> ServeStats:
    """Baseline: one request at a time, in arrival order, all its iterations
    before the next request starts."""
    stats = ServeStats()
    fake = isinstance(executor, FakeExecutor)
    for req in sorted(requests, key=lambda r: r.arrival):
        if fake:
            executor.t = max(executor.t, req.arrival)
        else:
            while executor.now() < req.arrival:
                time.sleep(min(0.01, req.arrival - executor.now()))
        adm = executor.now()
        h = executor.start(req, 0)
        while h["left"] > 0:
            if not executor.ready(h):
                if fake:
                    executor.advance([h])
                continue
            executor.step(h)
        if fake:
            executor.advance([h])
        x = executor.finish(h)
        stats.results.append(Result(req.rid, req.arrival, adm, executor.now(), x))
        stats.peak_active = 1
    stats.makespan = executor.now()
    stats.results.sort(key=lambda r: r.rid)
    return stats


# --------------------------------------------------------------------------- workload
def make_requests(n: int, rate: float, seed: int = 0, large_frac: float = 0.2, iters=(16, 32),
                  sizes=(64, 96, 128, 160), nzs=(32, 48, 64, 80, 96), views=(60, 90, 120, 128),
                  psfs=(11, 21, 29, 37), large=(192, 128, 128, 37), device=None, counts: float = 1e7,
                  background: float = 0.1):
    """Poisson arrivals of reconstructions of mixed sizes (synthetic phantoms).

    With ``device`` set, each request's measurements are simulated with the
    library's own projector: y ~ Poisson(A x_true + rbar), A x_true scaled to
    ``counts`` expected primary counts and rbar a uniform background carrying
    ``background`` of them (the paper's 10 % uniform scatter).  Without a
    device (scheduler tests on CPU) the counts are drawn around a constant mean.
    The large cases use the anisotropic depth-dependent PSF of the paper-scale
    workload, the others isotropic Gaussians with FWHM 1 -> 4 pixels.
    """
    from . import synthetic
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate)
        big = rng.uniform() < large_frac
        if big:
            nx, nz, nv, p = large
        else:
            nx, nz, nv, p = (int(rng.choice(sizes)), int(rng.choice(nzs)), int(rng.choice(views)),
                             int(rng.choice(psfs)))
        x, mu, body = synthetic.small_phantom(nx, nz, seed * 100003 + rid)
        if big:
            fx, fz = synthetic.depth_psf_factors(nx, p, p, 1.5, 9.0, aniso=True)
        else:
            fx, fz = synthetic.depth_psf_factors(nx, p, p, 1.0, 4.0, aniso=False)
        niter = int(rng.integers(iters[0], iters[1] + 1))
        if device is None:
            mean = np.full((nv, nz, nx), float(x.sum()) / (nz * nx) * 0.5 + 1.0, np.float32)
            y = rng.poisson(mean).astype(np.float32)
            rbar = np.full_like(y, 0.1 * float(mean.mean()))
        else:
            y, rbar = _simulate_counts(x, mu, fx, fz, nv, device, counts, background,
                                       np.random.default_rng([seed, rid]))
        reqs.append(Request(rid, t, nx, nz, nv, niter, mu, fx, fz, y, rbar,
                            np.where(body, 1.0, 0.0).astype(np.float32) + 0.01))
    return reqs


def _simulate_counts(x, mu, fx, fz, nview, device, counts, background, rng):
    """y ~ Poisson(A x + rbar) with A the library's projector for this geometry."""
    import torch

    from .projector import SpectPlan
    nz, nx, _ = x.shape
    plan = SpectPlan(nx, nz, nview, mu=mu, dy=1.0, fx=fx, fz=fz, device=device)
    primary = plan.forward(torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(device))
    plan.check()
    plan.close()
    primary = primary.double().cpu().numpy()
    primary *= counts / max(primary.sum(), 1e-30)
    rbar = np.full(primary.shape, background * primary.sum() / primary.size)
    y = rng.poisson(primary + rbar).astype(np.float32)
    return y, rbar.astype(np.float32)


def compare(requests, streams: int = 4, max_active: int = 8, iters_per_step: int = 2, device="cuda") -> dict:
    """Serve the requests with continuous batching, then one at a time through
    the same library calls; latency percentiles and throughput of both, and
    whether every request's image is bitwise the same in both runs."""
    ex = GpuExecutor(device=device, n_streams=streams, keep_images=True, iters_per_step=iters_per_step)
    st_served = serve(requests, ex, None, max_active)
    ex.close()
    ex2 = GpuExecutor(device=device, n_streams=1, keep_images=True, iters_per_step=iters_per_step)
    st_plain = serve_plain(requests, ex2)
    ex2.close()
    same = all(a.x is not None and np.array_equal(a.x, b.x) for a, b in zip(st_served.results, st_plain.results))
    return {"served": st_served.summary(), "plain": st_plain.summary(), "identical_images": bool(same)}


def main(argv=None):
    ap = argparse.ArgumentParser(description="serve EM reconstructions: continuous batching vs one at a time")
    ap.add_argument("--requests", type=int, default=60)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--max-active", type=int, default=8)
    ap.add_argument("--large-frac", type=float, default=0.2)
    a = ap.parse_args(argv)
    reqs = make_requests(a.requests, a.rate, large_frac=a.large_frac, device="cuda")
    print(json.dumps(compare(reqs, a.streams, a.max_active)))


if __name__ == "__main__":
    main()
