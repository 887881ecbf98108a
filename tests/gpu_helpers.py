"""Shared helpers for the GPU parity tests (CUDA path vs FP64 oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

REL_L2 = 2e-6      # relative L2 error bound of FP32 results vs the FP64 oracle
MAX_REL = 1e-4     # per-element bound, relative to max(|oracle|, 1e-3 max|oracle|)
ADJ_FP32 = 1e-5    # FP32 adjoint mismatch |<Ax,y> - <x,A'y>| / |<Ax,y>|


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def errors(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    rel_l2 = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)
    den = np.maximum(np.abs(want), 1e-3 * np.abs(want).max())
    max_rel = float(np.max(np.abs(got - want) / den)) if want.size else 0.0
    return rel_l2, max_rel


def assert_close(got, want, rel_l2=REL_L2, max_rel=MAX_REL, what=""):
    e2, emax = errors(got, want)
    assert e2 <= rel_l2 and emax <= max_rel, f"{what}: rel L2 {e2:.3e} (bound {rel_l2}), max rel {emax:.3e} (bound {max_rel})"
    return e2, emax


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


# the code paths of the library: fused kernels (separable PSF, default),
# low-memory kernels (separable PSF), fused full-PSF kernels, low-memory full-PSF kernels
PATHS = ["fused", "lowmem", "direct", "direct_lowmem"]


def make_plan(prob, angles, path, nview=None):
    """A plan of the given path; the tests call plan.check() through host() on it."""
    from paper_2301_09710_gb300 import SpectPlan
    nz, ny, nx = prob.x.shape
    nview = len(angles) if nview is None else nview
    if path in ("fused", "lowmem", True):
        return SpectPlan(nx, nz, nview, mu=prob.mu, dy=prob.dy, fx=prob.fx, fz=prob.fz, angles=angles,
                         low_memory=(path == "lowmem"))
    return SpectPlan(nx, nz, nview, mu=prob.mu, dy=prob.dy, psf=prob.full_psf(), angles=angles,
                     low_memory=(path == "direct_lowmem"))


def oracle_psf(prob, path):
    import oracle
    if path in ("fused", "lowmem", True):
        return oracle.psf_from_factors(prob.fx, prob.fz)
    return prob.full_psf().astype(np.float64)
