"""Python front end of the C ABI: a plan object over torch CUDA tensors.

Tensor layouts (C order, float32, contiguous, on the plan's CUDA device):
  x, mu : (nz, ny, nx)             x(i,j,k) = x[k, j, i]
  v, y  : (nview, nz, nx)          v(i,k,l) = v[l, k, i]
  psf   : (nview_psf, ny, pz, px)  p(a,b,j,l) = psf[l, j, b, a]
  fx    : (nview_psf, ny, px),  fz : (nview_psf, ny, pz)   p = fx (x) fz

Every method is argument marshalling around one C call (``include/spect.h``);
the work runs in the library's kernels on the current torch stream (or the
stream passed in).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib


def _as_dev(t, device) -> torch.Tensor:
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        t = torch.from_numpy(np.ascontiguousarray(np.asarray(t, dtype=np.float32)))
    return t.to(device=device, dtype=torch.float32).contiguous()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def fp32_peak(stream=None) -> dict:
    """Measured FP32 FMA throughput of the current device (TFLOP/s), scalar and packed."""
    lib = _lib.load()
    a, b = ctypes.c_double(), ctypes.c_double()
    _lib.check(lib.spect_fp32_peak(ctypes.byref(a), ctypes.byref(b), _stream_handle(stream)))
    return {"ffma_tflops": a.value, "ffma2_tflops": b.value}


def _ew_check(*ts):
    ref = next(t for t in ts if t is not None)
    for t in ts:
        if t is not None and (t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous()
                              or t.numel() != ref.numel() or t.device != ref.device):
            raise ValueError("element-wise EM arrays must be contiguous float32 CUDA tensors of one size and device")
    return ref.numel()


def em_ratio(ybar, y, rbar=None, out=None, stream=None):
    """ratio = y / (ybar + rbar), 0 where ybar + rbar <= 0 (spect_em_ratio)."""
    n = _ew_check(ybar, y, rbar)
    out = torch.empty_like(ybar) if out is None else out
    _ew_check(ybar, out)
    _lib.check(_lib.load().spect_em_ratio(n, _ptr(ybar), _ptr(y), _ptr(rbar), _ptr(out), _stream_handle(stream)))
    return out


def em_ratio_backward(ybar, y, rbar, g_ratio, stream=None):
    """dL/dybar of em_ratio from dL/dratio (spect_em_ratio_backward)."""
    n = _ew_check(ybar, y, rbar, g_ratio)
    out = torch.empty_like(ybar)
    _lib.check(_lib.load().spect_em_ratio_backward(n, _ptr(ybar), _ptr(y), _ptr(rbar), _ptr(g_ratio), _ptr(out),
                                                   _stream_handle(stream)))
    return out


def em_update(x, e, s, u=None, beta: float = 0.0, out=None, stream=None):
    """The EM update of Eqs. (7)-(8) from x, e = A'(ratio), s = A'1, u (spect_em_update)."""
    n = _ew_check(x, e, s, u if beta > 0 else None)
    out = torch.empty_like(x) if out is None else out
    _ew_check(x, out)
    _lib.check(_lib.load().spect_em_update(n, _ptr(x), _ptr(e), _ptr(s), _ptr(u if beta > 0 else None),
                                           ctypes.c_float(beta), _ptr(out), _stream_handle(stream)))
    return out


def em_update_backward(x, e, s, u, beta: float, g_out, stream=None):
    """(dL/dx, dL/de, dL/du) of em_update from dL/dout (spect_em_update_backward);
    dL/du is None when beta == 0."""
    n = _ew_check(x, e, s, g_out, u if beta > 0 else None)
    gx, ge = torch.empty_like(x), torch.empty_like(x)
    gu = torch.empty_like(x) if beta > 0 else None
    _lib.check(_lib.load().spect_em_update_backward(n, _ptr(x), _ptr(e), _ptr(s), _ptr(u if beta > 0 else None),
                                                    ctypes.c_float(beta), _ptr(g_out), _ptr(gx), _ptr(ge), _ptr(gu),
                                                    _stream_handle(stream)))
    return gx, ge, gu


def forward_static(x, nview: int, fx, fz, mu=None, dy: float = 1.0, angles=None, out=None, stream=None):
    """v = A x through spect_forward_static: no plan, no device allocation in
    the library (for callers that cannot allocate; see include/spect.h).

    x, mu: (nz, ny, nx); fx: (nview_psf, ny, px); fz: (nview_psf, ny, pz), all
    contiguous float32 CUDA tensors; out: (nview, nz, nx) or None (allocated
    here by torch, outside the library call).
    """
    lib = _lib.load()
    nz, ny, nx = x.shape
    nvp, _, px = fx.shape
    pz = fz.shape[-1]
    if out is None:
        out = torch.empty((nview, nz, nx), device=x.device, dtype=torch.float32)
    ang = None
    if angles is not None:
        a = np.ascontiguousarray(np.asarray(angles, dtype=np.float64))
        ang = a.ctypes.data_as(ctypes.c_void_p)
    _lib.check(lib.spect_forward_static(nx, ny, nz, int(nview), _ptr(x), _ptr(mu), ctypes.c_float(dy), _ptr(fx),
                                        _ptr(fz), px, pz, nvp, ang, _ptr(out), _stream_handle(stream)))
    return out


def _rotation_flag(rotation: str) -> int:
    if rotation not in _lib.ROTATIONS:
        raise ValueError(f"rotation must be one of {_lib.ROTATIONS}")
    return _lib.SPECT_PLAN_ROTATION_3PASS if rotation == "3pass" else 0


def plan_bytes(nx: int, nz: int, nview: int, px: int, pz: int, nview_psf: int = 1, separable: bool = True,
               low_memory: bool = False, rotation: str = "bilinear", recompute_attenuation: bool = False) -> int:
    """Upper bound of the device bytes a plan of this geometry allocates (no allocation)."""
    lib = _lib.load()
    out = ctypes.c_size_t()
    flags = (_lib.SPECT_PLAN_LOW_MEMORY if low_memory else 0) | _rotation_flag(rotation) | \
        (_lib.SPECT_PLAN_RECOMPUTE_ATTENUATION if recompute_attenuation else 0)
    _lib.check(lib.spect_plan_bytes(int(nx), int(nx), int(nz), int(nview), int(px), int(pz), int(nview_psf),
                                    int(bool(separable)), flags, ctypes.byref(out)))
    return out.value


class SpectPlan:
    """The operator A of one geometry (Algorithm 1 inputs) on one GPU.

    rotation: "bilinear" (default) or "3pass", the two image rotations of
    Section II-A (the three-pass one on the fused kernels only).
    recompute_attenuation: the fused kernels with the Eq. (1) factors made per
    view chunk instead of cached for every view (bitwise the same results,
    memory bounded by the chunk; SPECT_PLAN_RECOMPUTE_ATTENUATION).
    """

    def __init__(self, nx: int, nz: int, nview: int, mu=None, dy: float = 1.0, psf=None, fx=None, fz=None,
                 angles=None, prefer_separable: bool = True, low_memory: bool = False, device=None, stream=None,
                 rotation: str = "bilinear", recompute_attenuation: bool = False):
        self.lib = _lib.load()
        self.device = torch.device(device if device is not None else "cuda")
        self.nx = self.ny = int(nx)
        self.nz, self.nview = int(nz), int(nview)
        self._mu = _as_dev(mu, self.device)
        self._psf = _as_dev(psf, self.device)
        self._fx = _as_dev(fx, self.device)
        self._fz = _as_dev(fz, self.device)
        if self._psf is not None:
            nvp, _, pz, px = self._psf.shape
        else:
            nvp, _, px = self._fx.shape
            pz = self._fz.shape[-1]
        self.px, self.pz, self.nview_psf = int(px), int(pz), int(nvp)
        ang = None
        if angles is not None:
            self._angles = np.ascontiguousarray(np.asarray(angles, dtype=np.float64))
            ang = self._angles.ctypes.data_as(ctypes.c_void_p)
        handle = ctypes.c_void_p()
        flags = (_lib.SPECT_PLAN_PREFER_SEPARABLE if prefer_separable else 0) | \
            (_lib.SPECT_PLAN_LOW_MEMORY if low_memory else 0) | _rotation_flag(rotation) | \
            (_lib.SPECT_PLAN_RECOMPUTE_ATTENUATION if recompute_attenuation else 0)
        self.rotation = rotation
        with torch.cuda.device(self.device):
            _lib.check(self.lib.spect_plan_create(
                ctypes.byref(handle), self.nx, self.ny, self.nz, self.nview, _ptr(self._mu), ctypes.c_float(dy),
                _ptr(self._psf), _ptr(self._fx), _ptr(self._fz), self.px, self.pz, self.nview_psf, ang, flags,
                _stream_handle(stream)))
        self.handle = handle
        # the plan holds its own copies
        self._mu = self._psf = self._fx = self._fz = None

    # ------------------------------------------------------------------ shapes
    @property
    def vol_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def proj_shape(self):
        return (self.nview, self.nz, self.nx)

    def _check(self, t, shape, name):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")

    # ------------------------------------------------------------------ ops
    def forward(self, x, out=None, stream=None) -> torch.Tensor:
        """v = A x (Algorithm 1)."""
        self._check(x, self.vol_shape, "x")
        if out is None:
            out = torch.empty(self.proj_shape, device=x.device, dtype=torch.float32)
        self._check(out, self.proj_shape, "out")
        _lib.check(self.lib.spect_forward(self.handle, _ptr(x), _ptr(out), _stream_handle(stream)))
        return out

    def back(self, v, out=None, stream=None) -> torch.Tensor:
        """x = A' v (Algorithm 2), the exact transpose of forward()."""
        self._check(v, self.proj_shape, "v")
        if out is None:
            out = torch.empty(self.vol_shape, device=v.device, dtype=torch.float32)
        self._check(out, self.vol_shape, "out")
        _lib.check(self.lib.spect_back(self.handle, _ptr(v), _ptr(out), _stream_handle(stream)))
        return out

    def em_step(self, x, y, rbar=None, niter: int = 1, stream=None) -> torch.Tensor:
        """niter in-place MLEM updates x <- x A'(y/(Ax+rbar)) / A'1 (Eqs. (7)-(8), beta = 0)."""
        self._check(x, self.vol_shape, "x")
        self._check(y, self.proj_shape, "y")
        if rbar is not None:
            self._check(rbar, self.proj_shape, "rbar")
        _lib.check(self.lib.spect_em_step(self.handle, _ptr(x), _ptr(y), _ptr(rbar), int(niter),
                                          _stream_handle(stream)))
        return x

    def em_step_reg(self, x, y, u, beta: float, rbar=None, niter: int = 1, stream=None) -> torch.Tensor:
        """niter in-place regularised EM updates (Eqs. (7)-(8)) towards u with weight beta."""
        self._check(x, self.vol_shape, "x")
        self._check(y, self.proj_shape, "y")
        if u is not None:
            self._check(u, self.vol_shape, "u")
        if rbar is not None:
            self._check(rbar, self.proj_shape, "rbar")
        _lib.check(self.lib.spect_em_step_reg(self.handle, _ptr(x), _ptr(y), _ptr(rbar), _ptr(u),
                                              ctypes.c_float(beta), int(niter), _stream_handle(stream)))
        return x

    def sensitivity(self, stream=None) -> torch.Tensor:
        """s = A' 1."""
        s = torch.empty(self.vol_shape, device=self.device, dtype=torch.float32)
        _lib.check(self.lib.spect_sensitivity(self.handle, _ptr(s), _stream_handle(stream)))
        return s

    def info(self) -> dict:
        """separable: separable-factor kernels; view_chunk: views per slab pass; device_bytes: plan memory."""
        sep, fused, chunk = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nbytes = ctypes.c_size_t()
        _lib.check(self.lib.spect_plan_info(self.handle, ctypes.byref(sep), ctypes.byref(fused), ctypes.byref(chunk),
                                            ctypes.byref(nbytes)))
        return {"separable": bool(sep.value), "fused": bool(fused.value), "view_chunk": chunk.value,
                "device_bytes": nbytes.value}

    def check(self, stream=None) -> None:
        """Synchronise (the device, or only ``stream`` when given) and raise
        SpectError(SPECT_ETIMEOUT) if a bounded device wait ran out."""
        if stream is not None:
            _lib.check(self.lib.spect_plan_check_stream(self.handle, _stream_handle(stream)))
        else:
            _lib.check(self.lib.spect_plan_check(self.handle))

    def selftest_timeout(self, spin_clocks: int = 1 << 22, stream=None) -> None:
        """Make one bounded device wait run out (nothing completes it): the next
        check() raises SpectError(SPECT_ETIMEOUT); the plan stays usable."""
        _lib.check(self.lib.spect_plan_selftest_timeout(self.handle, int(spin_clocks), _stream_handle(stream)))

    def profile(self, enable: bool = True) -> None:
        """Bracket every later kernel launch with CUDA events on its stream."""
        _lib.check(self.lib.spect_profile_enable(self.handle, int(bool(enable))))

    def profile_read(self, reset: bool = False) -> dict:
        """{kernel class: (launches, summed device ms)} since the last reset."""
        n = len(_lib.KERNEL_CLASSES)
        la = (ctypes.c_longlong * n)()
        ms = (ctypes.c_double * n)()
        _lib.check(self.lib.spect_profile_read(self.handle, la, ms, int(bool(reset))))
        return {k: (la[i], ms[i]) for i, k in enumerate(_lib.KERNEL_CLASSES)}

    # ------------------------------------------------------------------ launch shapes
    @property
    def tuning(self) -> dict:
        """fused_J / adj_J: depth planes per forward / adjoint blur block; tiles: column tiles per plane."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.check(self.lib.spect_plan_get_tuning(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"fused_J": a.value, "adj_J": b.value, "tiles": c.value}

    def set_tuning(self, fused_J: int, adj_J: int, tiles: int, stream=None) -> None:
        _lib.check(self.lib.spect_plan_set_tuning(self.handle, int(fused_J), int(adj_J), int(tiles),
                                                  _stream_handle(stream)))

    def autotune(self, stream=None) -> dict:
        """Time the candidate launch shapes on this device and keep the fastest (cached per geometry)."""
        _lib.check(self.lib.spect_plan_autotune(self.handle, _stream_handle(stream)))
        return self.tuning

    def release(self, stream) -> None:
        """Free the plan after the work already enqueued on ``stream``, without
        waiting for the device (all of the plan's work must be on ``stream``)."""
        if getattr(self, "handle", None) is not None and self.handle.value:
            h, self.handle = self.handle, None
            _lib.check(self.lib.spect_plan_release(h, _stream_handle(stream)))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.check(self.lib.spect_plan_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class SpectBatch:
    """Plans of different sizes whose EM iterations run as one CUDA graph launch:
    one graph branch per plan (grouped=0), or grouped launches -- one per stage and
    kernel variant over the blocks of every plan -- in `grouped` branches
    (spect_batch_em_step, spect_batch_set_grouped)."""

    def __init__(self, plans, grouped: int = 0):
        self.lib = _lib.load()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        handle = ctypes.c_void_p()
        _lib.check(self.lib.spect_batch_create(ctypes.byref(handle), arr, len(self.plans)))
        self.handle = handle
        if grouped:
            self.set_grouped(grouped)

    def set_grouped(self, branches: int) -> None:
        _lib.check(self.lib.spect_batch_set_grouped(self.handle, int(branches)))

    def em_step(self, xs, ys, rbars=None, niter: int = 1, stream=None):
        """niter MLEM updates of every plan's x in place (xs, ys, rbars: lists of CUDA tensors)."""
        n = len(self.plans)
        if len(xs) != n or len(ys) != n or (rbars is not None and len(rbars) != n):
            raise ValueError("one x, y (and rbar) per plan")
        for p, x, y in zip(self.plans, xs, ys):
            p._check(x, p.vol_shape, "x")
            p._check(y, p.proj_shape, "y")
        if rbars is not None:
            for p, r in zip(self.plans, rbars):
                if r is not None:
                    p._check(r, p.proj_shape, "rbar")
        P = ctypes.c_void_p * n
        xa = P(*[x.data_ptr() for x in xs])
        ya = P(*[y.data_ptr() for y in ys])
        ra = P(*[(r.data_ptr() if r is not None else None) for r in rbars]) if rbars is not None else None
        _lib.check(self.lib.spect_batch_em_step(self.handle, xa, ya, ra, int(niter), _stream_handle(stream)))
        return xs

    def info(self) -> dict:
        n, k = ctypes.c_int(), ctypes.c_longlong()
        _lib.check(self.lib.spect_batch_info(self.handle, ctypes.byref(n), ctypes.byref(k)))
        return {"plans": n.value, "kernels_per_launch": k.value}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.check(self.lib.spect_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
