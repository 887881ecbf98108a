"""OSEM on the GPU (each sub-iteration one library EM step over the subset's
plan) against the oracle's OSEM iteration."""
import numpy as np
import pytest

import oracle
from paper_2301_09710_gb300 import synthetic

from gpu_helpers import assert_close, dev, host, need_gpu, oracle_psf, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("case", [(32, 12, 16, 7, 4, False), (24, 8, 12, 5, 3, True), (33, 10, 9, 9, 1, False)],
                         ids=["32x12v16s4", "24x8v12s3-viewpsf", "33x10v9s1"])
def test_osem_matches_oracle(case):
    from paper_2301_09710_gb300.osem import OSEM
    nx, nz, nview, p, M, per_view = case
    prob = synthetic.random_problem(50 + M, nx=nx, nz=nz, nview=nview, px=p, pz=p,
                                    nview_psf=nview if per_view else 1, mu_scale=0.1)
    ang = oracle.default_angles(nview)
    psf = oracle_psf(prob, "fused")
    y = synthetic.poisson_counts(oracle.forward(prob.x, prob.mu, psf, prob.dy, ang) * 30, 5)
    rbar = np.full_like(y, 0.2)
    os_ = OSEM(nx, nz, nview, M, mu=prob.mu, dy=prob.dy, fx=prob.fx, fz=prob.fz, angles=ang)
    x0 = np.full(prob.x.shape, 0.5, np.float32)
    xg = dev(x0)
    os_.step(xg, os_.split(dev(y)), os_.split(dev(rbar)), niter=1)
    want = oracle.osem_step(x0, y, rbar, prob.mu, psf, prob.dy, ang, M)
    # M sequential EM updates: the FP32 error of one update (2e-6) compounds over the subsets
    assert_close(host(xg), want, rel_l2=2e-6 * M, max_rel=1e-4 * M, what=f"OSEM, {M} subsets")
    os_.check()
    os_.close()
