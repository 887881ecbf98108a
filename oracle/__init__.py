"""FP64 CPU oracle for the rotation-based SPECT projector (arXiv 2301.09710).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The product library (``paper_2301_09710_gb300``) never imports it, and the
two share no code: the only module both sides use is the seeded input
generator ``paper_2301_09710_gb300.synthetic``, which holds none of the
method's arithmetic.

The projector steps (rotation, Eq. (1) attenuation, PSF blur with replicate
padding, depth sum, and their transposes) are plain C loops in
``spect_oracle.c``; this module marshals numpy arrays to it and writes the
EM update (Eqs. (7)-(8) with beta = 0, i.e. MLEM) in numpy on top of it.

Array layouts (numpy, C order):
  x, mu  : shape (nz, ny, nx)            -> x(i,j,k) = x[k, j, i]
  psf    : shape (nview_psf, ny, pz, px) -> p(a,b,j,l) = psf[l, j, b, a]
  v      : shape (nview, nz, nx)         -> v(i,k,l) = v[l, k, i]

Parity of the reconstruction results with the authors' Julia package is
unpinned (that code is not available); the operator itself is pinned by the
tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spect_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libspect_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile spect_oracle.c with gcc (OpenMP) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            i = ctypes.c_int
            d = ctypes.c_double
            lib.oracle_rotate_slice.argtypes = [i, d, dp, dp]
            lib.oracle_rotate_adjoint_slice.argtypes = [i, d, dp, dp]
            lib.oracle_rotate3_slice.argtypes = [i, d, dp, dp]
            lib.oracle_rotate3_adjoint_slice.argtypes = [i, d, dp, dp]
            lib.oracle_attenuation.argtypes = [i, i, i, d, dp, dp]
            lib.oracle_conv_plane.argtypes = [i, i, dp, dp, i, i, dp]
            lib.oracle_conv_adjoint_plane.argtypes = [i, i, dp, dp, i, i, dp]
            lib.oracle_forward.argtypes = [i, i, i, i, dp, dp, d, dp, i, i, i, dp, dp, i, i]
            lib.oracle_back.argtypes = [i, i, i, i, dp, dp, d, dp, i, i, i, dp, dp, i, i]
            lib.oracle_max_threads.restype = i
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def default_angles(nview: int) -> np.ndarray:
    """theta_l = 2*pi*(l-1)/nview for the paper's 1-based l (Section II-A)."""
    return 2.0 * np.pi * np.arange(nview, dtype=np.float64) / nview


# ---------------------------------------------------------------- single steps
def rotate_slice(img2d, theta: float) -> np.ndarray:
    """Bilinear rotation of one (ny, nx) slice by theta, zero padding."""
    a = _f64(img2d)
    n = a.shape[0]
    assert a.shape == (n, n)
    out = np.empty_like(a)
    _load().oracle_rotate_slice(n, float(theta), _ptr(a), _ptr(out))
    return out


def rotate_adjoint_slice(img2d, theta: float) -> np.ndarray:
    """Transpose of :func:`rotate_slice` (scatter form)."""
    a = _f64(img2d)
    n = a.shape[0]
    out = np.empty_like(a)
    _load().oracle_rotate_adjoint_slice(n, float(theta), _ptr(a), _ptr(out))
    return out


def rotate3_slice(img2d, theta: float) -> np.ndarray:
    """Three-pass rotation of one (ny, nx) slice by theta: the exact quarter turn,
    then 1D linear interpolation along x, y, x (zero padding), reading R13."""
    a = _f64(img2d)
    n = a.shape[0]
    assert a.shape == (n, n)
    out = np.empty_like(a)
    _load().oracle_rotate3_slice(n, float(theta), _ptr(a), _ptr(out))
    return out


def rotate3_adjoint_slice(img2d, theta: float) -> np.ndarray:
    """Transpose of :func:`rotate3_slice` (scatter form, passes in reverse order)."""
    a = _f64(img2d)
    n = a.shape[0]
    out = np.empty_like(a)
    _load().oracle_rotate3_adjoint_slice(n, float(theta), _ptr(a), _ptr(out))
    return out


ROTATIONS = {"bilinear": 0, "3pass": 1}


def attenuation(mu_rot, dy: float) -> np.ndarray:
    """Eq. (1) accumulated attenuation of a rotated-frame map (nz, ny, nx)."""
    m = _f64(mu_rot)
    nz, ny, nx = m.shape
    out = np.empty_like(m)
    _load().oracle_attenuation(nx, ny, nz, float(dy), _ptr(m), _ptr(out))
    return out


def conv_plane(w, p) -> np.ndarray:
    """Replicate-padded true convolution of one (nz, nx) plane with p (pz, px)."""
    w = _f64(w)
    p = _f64(p)
    nz, nx = w.shape
    pz, px = p.shape
    out = np.empty_like(w)
    _load().oracle_conv_plane(nx, nz, _ptr(w), _ptr(p), px, pz, _ptr(out))
    return out


def conv_adjoint_plane(v, p) -> np.ndarray:
    """Transpose of :func:`conv_plane` (scatter form)."""
    v = _f64(v)
    p = _f64(p)
    nz, nx = v.shape
    pz, px = p.shape
    out = np.empty_like(v)
    _load().oracle_conv_adjoint_plane(nx, nz, _ptr(v), _ptr(p), px, pz, _ptr(out))
    return out


def psf_from_factors(fx, fz) -> np.ndarray:
    """Full PSF stack from separable factors: p(a,b,j,l) = fx(a,j,l) fz(b,j,l).

    fx: (nview_psf, ny, px), fz: (nview_psf, ny, pz) -> (nview_psf, ny, pz, px).
    The products of FP32 inputs are exact in FP64.
    """
    fx = _f64(fx)
    fz = _f64(fz)
    return fz[..., :, None] * fx[..., None, :]


# ---------------------------------------------------------------- projectors
def _check(x_shape, mu, psf, angles):
    nz, ny, nx = x_shape
    assert nx == ny, "rotation about the axial axis needs nx == ny"
    assert mu.shape == (nz, ny, nx)
    assert psf.ndim == 4 and psf.shape[1] == ny
    nview_psf, _, pz, px = psf.shape
    assert px % 2 == 1 and pz % 2 == 1
    nview = len(angles)
    assert nview_psf in (1, nview)
    return nx, ny, nz, nview, px, pz, nview_psf


def forward(x, mu, psf, dy: float, angles, nthreads: int = 0, rotation: str = "bilinear") -> np.ndarray:
    """v = A x, Algorithm 1.  Returns (nview, nz, nx) float64.  rotation: "bilinear"
    (R1, R2) or "3pass" (R13), the two image rotations of Section II-A."""
    x = _f64(x)
    mu = _f64(mu)
    psf = _f64(psf)
    angles = _f64(angles)
    nx, ny, nz, nview, px, pz, nvp = _check(x.shape, mu, psf, angles)
    v = np.empty((nview, nz, nx), dtype=np.float64)
    _load().oracle_forward(nx, ny, nz, nview, _ptr(x), _ptr(mu), float(dy), _ptr(psf), px, pz, nvp,
                           _ptr(angles), _ptr(v), int(nthreads), ROTATIONS[rotation])
    return v


def back(v, mu, psf, dy: float, angles, nthreads: int = 0, rotation: str = "bilinear") -> np.ndarray:
    """x = A' v, Algorithm 2 (literal transpose of :func:`forward`)."""
    v = _f64(v)
    mu = _f64(mu)
    psf = _f64(psf)
    angles = _f64(angles)
    nz, ny, nx = mu.shape
    nx_, ny_, nz_, nview, px, pz, nvp = _check((nz, ny, nx), mu, psf, angles)
    assert v.shape == (nview, nz, nx)
    x = np.empty((nz, ny, nx), dtype=np.float64)
    _load().oracle_back(nx, ny, nz, nview, _ptr(v), _ptr(mu), float(dy), _ptr(psf), px, pz, nvp,
                        _ptr(angles), _ptr(x), int(nthreads), ROTATIONS[rotation])
    return x


def sensitivity(mu, psf, dy: float, angles, nthreads: int = 0, rotation: str = "bilinear") -> np.ndarray:
    """s = A' 1 (the EM normaliser d(0) of Eq. (8))."""
    nz, ny, nx = np.shape(mu)
    ones = np.ones((len(angles), nz, nx), dtype=np.float64)
    return back(ones, mu, psf, dy, angles, nthreads, rotation)


def em_step(x, y, rbar, mu, psf, dy: float, angles, s=None, nthreads: int = 0,
            rotation: str = "bilinear") -> np.ndarray:
    """One MLEM update, Eqs. (7)-(8) with beta = 0:

        x+ = x * A'(y / (A x + rbar)) / A'1.

    Guards (the paper states none): where A x + rbar <= 0 the ratio is 0,
    and where A'1 <= 0 the voxel is set to 0.
    """
    x = _f64(x)
    y = _f64(y)
    if s is None:
        s = sensitivity(mu, psf, dy, angles, nthreads, rotation)
    ybar = forward(x, mu, psf, dy, angles, nthreads, rotation)
    if rbar is not None:
        ybar = ybar + _f64(rbar)
    ratio = np.zeros_like(ybar)
    pos = ybar > 0
    ratio[pos] = y[pos] / ybar[pos]
    e = back(ratio, mu, psf, dy, angles, nthreads, rotation)
    out = np.zeros_like(x)
    ok = s > 0
    out[ok] = x[ok] * e[ok] / s[ok]
    return out


def em_ratio(ybar, y, rbar=None) -> np.ndarray:
    """The ratio y / (ybar + rbar) of Eq. (8), 0 where ybar + rbar <= 0 (the guard of em_step)."""
    yb = _f64(ybar) + (0.0 if rbar is None else _f64(rbar))
    out = np.zeros_like(yb)
    pos = yb > 0
    out[pos] = _f64(y)[pos] / yb[pos]
    return out


def em_ratio_vjp(ybar, y, rbar, g) -> np.ndarray:
    """dL/dybar of em_ratio given dL/dratio: d(y/(ybar + rbar))/dybar = -y/(ybar + rbar)^2."""
    yb = _f64(ybar) + (0.0 if rbar is None else _f64(rbar))
    out = np.zeros_like(yb)
    pos = yb > 0
    out[pos] = -_f64(g)[pos] * _f64(y)[pos] / yb[pos] ** 2
    return out


def em_root(x, e, s, u, beta: float) -> np.ndarray:
    """The update of Eqs. (7)-(8) from x_k, e = A'(y / (A x_k + rbar)), s = A'1 and u:
    the non-negative root of beta x^2 + d x - x_k e = 0, d = s - beta u.  beta = 0: the
    MLEM update x e / s (0 where s <= 0).  beta > 0: where d >= 0 the root is
    written 2 x e / (d + sqrt(d^2 + 4 beta x e)) (no cancellation for small beta),
    where d < 0 as (sqrt(d^2 + 4 beta x e) - d) / (2 beta); 0 where the denominator
    is not positive."""
    x = _f64(x)
    e = _f64(e)
    s = _f64(s)
    xe = x * e
    out = np.zeros_like(x)
    if beta == 0:
        ok = s > 0
        out[ok] = xe[ok] / s[ok]
        return out
    d = s - beta * _f64(u)
    root = np.sqrt(d * d + 4.0 * beta * xe)
    pos = d >= 0
    den = d + root
    ok = pos & (den > 0)
    out[ok] = 2.0 * xe[ok] / den[ok]
    neg = ~pos
    out[neg] = (root[neg] - d[neg]) / (2.0 * beta)
    return out


def em_root_vjp(x, e, s, u, beta: float, g):
    """(dL/dx, dL/de, dL/du) of em_root given dL/dx+.  Differentiating
    beta x+^2 + d x+ - x e = 0 (d = s - beta u) implicitly:
    (2 beta x+ + d) dx+ = e dx + x de + beta x+ du, with 2 beta x+ + d =
    sqrt(d^2 + 4 beta x e) = q; at beta = 0, x+ = x e / s and q = s.  Zero where
    em_root's guard set x+ to 0."""
    x = _f64(x)
    e = _f64(e)
    s = _f64(s)
    g = _f64(g)
    gx, ge, gu = np.zeros_like(x), np.zeros_like(x), np.zeros_like(x)
    if beta == 0:
        ok = s > 0
        gx[ok] = g[ok] * e[ok] / s[ok]
        ge[ok] = g[ok] * x[ok] / s[ok]
        return gx, ge, gu
    d = s - beta * _f64(u)
    q = np.sqrt(d * d + 4.0 * beta * x * e)
    ok = ((d < 0) | (d + q > 0)) & (q > 0)
    xp = em_root(x, e, s, u, beta)
    gx[ok] = g[ok] * e[ok] / q[ok]
    ge[ok] = g[ok] * x[ok] / q[ok]
    gu[ok] = g[ok] * beta * xp[ok] / q[ok]
    return gx, ge, gu


def em_step_reg(x, y, rbar, u, beta: float, mu, psf, dy: float, angles, s=None, nthreads: int = 0) -> np.ndarray:
    """One inner iteration of the regularised EM update, Eqs. (7)-(8):

        x+ = (-d + sqrt(d^2 + 4 beta x e)) / (2 beta),
        d = A'1 - beta u,   e = A'(y / (A x + rbar)),

    the non-negative root of beta x^2 + d x - x_k e = 0 (the EM surrogate of
    Eq. (6) with the penalty (beta/2)||x - u||^2).  Where d >= 0 it is written
    as 2 x e / (d + sqrt(d^2 + 4 beta x e)) (no cancellation for small beta;
    equals the MLEM update x e / A'1 at beta = 0), where d < 0 as Eq. (7)
    itself (no cancellation there).
    Guards as em_step: ratio 0 where A x + rbar <= 0; voxel 0 where the
    result is not finite and positive.
    """
    x = _f64(x)
    y = _f64(y)
    u = _f64(u)
    if s is None:
        s = sensitivity(mu, psf, dy, angles, nthreads)
    ybar = forward(x, mu, psf, dy, angles, nthreads)
    if rbar is not None:
        ybar = ybar + _f64(rbar)
    ratio = np.zeros_like(ybar)
    pos = ybar > 0
    ratio[pos] = y[pos] / ybar[pos]
    e = back(ratio, mu, psf, dy, angles, nthreads)
    return em_root(x, e, s, u, beta)


def poisson_loglik(x, y, rbar, mu, psf, dy: float, angles, nthreads: int = 0) -> float:
    """-f(x) of Eq. (4) (up to the constant log y!): y' log(Ax + r) - 1'(Ax + r)."""
    ybar = forward(x, mu, psf, dy, angles, nthreads)
    if rbar is not None:
        ybar = ybar + _f64(rbar)
    y = _f64(y)
    pos = y > 0
    return float(np.sum(y[pos] * np.log(ybar[pos])) - np.sum(ybar))


def osem_subsets(nview: int, n_subsets: int) -> list:
    """View indices of each ordered subset: subset m holds the views l = m (mod M),
    interleaved over the orbit (the paper runs OSEM with 4 subsets and does not
    say how they are formed; interleaving is the usual choice)."""
    if not 1 <= n_subsets <= nview:
        raise ValueError("need 1 <= n_subsets <= nview")
    return [np.arange(m, nview, n_subsets) for m in range(n_subsets)]


def osem_step(x, y, rbar, mu, psf, dy: float, angles, n_subsets: int, nthreads: int = 0) -> np.ndarray:
    """One OSEM iteration (the EM update of Eqs. (7)-(8), beta = 0, applied in turn
    to each ordered subset of views with that subset's projector and sensitivity):

        x <- x * A_S'(y_S / (A_S x + rbar_S)) / A_S'1   for S = S_0, ..., S_{M-1}.

    psf with one view row (nview_psf = 1) serves every subset; otherwise the
    subset's rows are taken.  Guards as em_step.  With M = 1 this is em_step.
    """
    x = _f64(x)
    y = _f64(y)
    angles = np.asarray(angles, dtype=np.float64)
    psf = _f64(psf)
    for idx in osem_subsets(len(angles), n_subsets):
        p = psf if psf.shape[0] == 1 else psf[idx]
        r = None if rbar is None else _f64(rbar)[idx]
        x = em_step(x, y[idx], r, mu, p, dy, angles[idx], nthreads=nthreads)
    return x
