"""Differentiation through the projector and the unrolled CNN-regularised EM.

* the autograd Jacobians of A and A' against the FP64 oracle gradient;
* the fused regularised EM update (Eqs. (7)-(8), beta > 0) against the oracle;
* the unrolled network's parameter gradient against central finite differences
  (16x16x8, 8 views, 5x5 PSF) and against the same network run in FP64 on the
  oracle (CPU autograd with oracle-backed A / A').
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


def _small():
    prob = synthetic.config1(seed=5, nx=16, nz=8, nview=8, psf_size=5)
    ang = oracle.default_angles(8)
    return prob, ang


@pytest.mark.parametrize("path", ["fused", "lowmem"])
def test_least_squares_gradient_matches_oracle(path):
    from paper_2301_09710_gb300.autograd import backproject, project
    prob, ang = _small()
    plan = make_plan(prob, ang, path)
    psf = oracle_psf(prob, path)
    rng = np.random.default_rng(3)
    y = (oracle.forward(prob.x, prob.mu, psf, prob.dy, ang) + rng.normal(0, 0.5, plan.proj_shape)).astype(np.float32)
    x = dev(prob.x + 0.3).requires_grad_(True)
    loss = 0.5 * ((project(x, plan) - dev(y)) ** 2).sum()
    loss.backward()
    xo = (prob.x + 0.3).astype(np.float32)
    g_o = oracle.back(oracle.forward(xo, prob.mu, psf, prob.dy, ang) - y, prob.mu, psf, prob.dy, ang)
    assert_close(host(x.grad), g_o, rel_l2=1e-5, max_rel=1e-3, what="grad of 0.5|Ax-y|^2")
    # and the backward of A' is A
    v = dev(y).requires_grad_(True)
    (backproject(v, plan) * x.detach()).sum().backward()
    assert_close(host(v.grad), oracle.forward(xo, prob.mu, psf, prob.dy, ang), what="grad through A'")


@pytest.mark.parametrize("path", ["fused", "lowmem"])
def test_regularised_em_step_matches_oracle(path):
    prob, ang = _small()
    plan = make_plan(prob, ang, path)
    psf = oracle_psf(prob, path)
    rng = np.random.default_rng(4)
    ybar = oracle.forward(prob.x, prob.mu, psf, prob.dy, ang)
    y = synthetic.poisson_counts(ybar * 50, 2)
    rbar = np.full_like(y, 0.1 * y.mean())
    x0 = np.where(prob.body, 1.0, 0.0).astype(np.float32) + 0.1
    u = rng.uniform(0.2, 3.0, x0.shape).astype(np.float32)
    for beta in (0.05, 5.0):
        xg = dev(x0)
        plan.em_step_reg(xg, dev(y), dev(u), beta, rbar=dev(rbar), niter=1)
        want = oracle.em_step_reg(x0, y, rbar, u, beta, prob.mu, psf, prob.dy, ang)
        assert_close(host(xg), want, what=f"regularised EM, beta={beta}")
    plan.check()


def _unrolled(plan, dtype=torch.float32, device="cuda"):
    from paper_2301_09710_gb300.autograd import Regularizer3D, UnrolledEM
    torch.manual_seed(0)
    cnn = Regularizer3D(channels=4).to(device=device, dtype=dtype)
    with torch.no_grad():
        for p in cnn.parameters():
            p.normal_(0, 0.05)
    return UnrolledEM(plan, n_outer=2, n_inner=1, beta=0.5, cnn=cnn)


def test_unrolled_em_gradient_finite_differences():
    prob, ang = _small()
    plan = make_plan(prob, ang, "fused")
    psf = oracle_psf(prob, "fused")
    y = synthetic.poisson_counts(oracle.forward(prob.x, prob.mu, psf, prob.dy, ang) * 20, 3)
    target = dev(prob.x * 20)
    net = _unrolled(plan)
    x0, yd = dev(np.ones_like(prob.x)), dev(y)

    def loss_fn():
        return ((net(x0, yd) - target) ** 2).mean()

    loss = loss_fn()
    loss.backward()
    params = list(net.cnn.parameters())
    rng = np.random.default_rng(7)
    # a probe direction on the scale of the weights, small enough that ReLU
    # patterns and the update's branches do not change
    dirs = [torch.from_numpy(rng.normal(0, 0.05, p.shape).astype(np.float32)).cuda() for p in params]
    g_dot = sum((p.grad * d).sum().item() for p, d in zip(params, dirs))

    def central(eps):
        with torch.no_grad():
            for p, d in zip(params, dirs):
                p.add_(eps * d)
            lp = loss_fn().item()
            for p, d in zip(params, dirs):
                p.add_(-2 * eps * d)
            lm = loss_fn().item()
            for p, d in zip(params, dirs):
                p.add_(eps * d)
        return (lp - lm) / (2 * eps)

    # Richardson-extrapolated central difference; the loss is evaluated in FP32,
    # so this is a coarse check (the tight one is the FP64 oracle network below)
    fd = (4 * central(1e-2) - central(2e-2)) / 3
    assert abs(fd - g_dot) <= 5e-2 * abs(g_dot) + 1e-6, (fd, g_dot)


class _OracleProject(torch.autograd.Function):
    """A on the FP64 oracle (CPU), backward A' -- test infrastructure only."""

    @staticmethod
    def forward(ctx, x, args):
        ctx.args = args
        mu, psf, dy, ang = args
        return torch.from_numpy(oracle.forward(x.detach().numpy(), mu, psf, dy, ang))

    @staticmethod
    def backward(ctx, g):
        mu, psf, dy, ang = ctx.args
        return torch.from_numpy(oracle.back(g.detach().numpy(), mu, psf, dy, ang)), None


class _OracleBack(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, args):
        ctx.args = args
        mu, psf, dy, ang = args
        return torch.from_numpy(oracle.back(v.detach().numpy(), mu, psf, dy, ang))

    @staticmethod
    def backward(ctx, g):
        mu, psf, dy, ang = ctx.args
        return torch.from_numpy(oracle.forward(g.detach().numpy(), mu, psf, dy, ang)), None


def test_unrolled_em_gradient_matches_fp64_oracle_network(monkeypatch):
    import paper_2301_09710_gb300.autograd as ag
    from test_autograd_cpu import use_oracle_em
    prob, ang = _small()
    plan = make_plan(prob, ang, "fused")
    psf = oracle_psf(prob, "fused")
    y = synthetic.poisson_counts(oracle.forward(prob.x, prob.mu, psf, prob.dy, ang) * 20, 3)
    target = prob.x * 20
    # GPU FP32
    net = _unrolled(plan)
    loss = ((net(dev(np.ones_like(prob.x)), dev(y)) - dev(target)) ** 2).mean()
    loss.backward()
    g_gpu = [host(p.grad) for p in net.cnn.parameters()]
    # CPU FP64 with the oracle as A / A' and the same weights
    args = (prob.mu, psf, prob.dy, ang)
    monkeypatch.setattr(ag, "project", lambda x, plan: _OracleProject.apply(x, args))
    monkeypatch.setattr(ag, "backproject", lambda v, plan: _OracleBack.apply(v, args))
    use_oracle_em(monkeypatch)
    net64 = _unrolled(None, dtype=torch.float64, device="cpu")
    net64.cnn.load_state_dict({k: v.double().cpu() for k, v in net.cnn.state_dict().items()})
    net64._s = torch.from_numpy(oracle.sensitivity(prob.mu, psf, prob.dy, ang))
    loss64 = ((net64(torch.ones(prob.x.shape, dtype=torch.float64), torch.from_numpy(y.astype(np.float64)))
               - torch.from_numpy(target.astype(np.float64))) ** 2).mean()
    loss64.backward()
    g_cpu = [p.grad.numpy() for p in net64.cnn.parameters()]
    assert abs(loss.item() - loss64.item()) <= 1e-5 * abs(loss64.item())
    for a, b in zip(g_gpu, g_cpu):
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b) + 1e-9


# ---------------------------------------------------------------- element-wise EM kernels and their gradients
@pytest.mark.parametrize("beta", [0.0, 0.05, 0.7, 30.0])
def test_em_update_kernels_match_oracle(beta):
    """spect_em_update / spect_em_update_backward against the oracle's closed-form
    root and its implicit derivatives (FP64), element by element, with d = s - beta u
    of both signs and a few voxels on the guards (s <= 0, x e = 0)."""
    from paper_2301_09710_gb300 import projector as pj
    rng = np.random.default_rng(41)
    n = 4099  # not a multiple of 4: the scalar path
    x, e = rng.uniform(0.2, 3.0, n), rng.uniform(0.2, 3.0, n)
    s, u, g = rng.uniform(0.5, 2.0, n), rng.uniform(0.0, 4.0, n), rng.normal(0, 1, n)
    x[:5], e[5:10], s[10:15] = 0.0, 0.0, 0.0
    f32 = [a.astype(np.float32) for a in (x, e, s, u, g)]
    xd, ed, sd, ud, gd = (dev(a) for a in f32)
    got = host(pj.em_update(xd, ed, sd, ud, beta))
    x64, e64, s64, u64, g64 = (a.astype(np.float64) for a in f32)
    want = oracle.em_root(x64, e64, s64, u64, beta)
    assert_close(got, want, rel_l2=1e-6, max_rel=1e-5, what=f"EM update, beta={beta}")
    gx, ge, gu = pj.em_update_backward(xd, ed, sd, ud, beta, gd)
    wx, we, wu = oracle.em_root_vjp(x64, e64, s64, u64, beta, g64)
    assert_close(host(gx), wx, rel_l2=1e-6, max_rel=1e-5, what=f"dL/dx, beta={beta}")
    assert_close(host(ge), we, rel_l2=1e-6, max_rel=1e-5, what=f"dL/de, beta={beta}")
    if beta > 0:
        assert_close(host(gu), wu, rel_l2=1e-6, max_rel=1e-5, what=f"dL/du, beta={beta}")
    else:
        assert gu is None


@pytest.mark.parametrize("n", [4096, 4097])
def test_em_ratio_kernels_match_oracle(n):
    from paper_2301_09710_gb300 import projector as pj
    rng = np.random.default_rng(42)
    ybar, y = rng.uniform(0.1, 5.0, n), rng.poisson(3.0, n).astype(np.float64)
    rbar, g = rng.uniform(0.0, 0.5, n), rng.normal(0, 1, n)
    ybar[:7] = -1.0  # ybar + rbar <= 0: ratio and gradient 0
    f32 = [a.astype(np.float32) for a in (ybar, y, rbar, g)]
    yb, yd, rd, gd = (dev(a) for a in f32)
    b64 = [a.astype(np.float64) for a in f32]
    assert_close(host(pj.em_ratio(yb, yd, rd)), oracle.em_ratio(*b64[:3]), rel_l2=1e-6, max_rel=1e-5,
                 what="EM ratio")
    assert_close(host(pj.em_ratio_backward(yb, yd, rd, gd)), oracle.em_ratio_vjp(*b64), rel_l2=1e-6, max_rel=1e-5,
                 what="EM ratio gradient")
    assert host(pj.em_ratio(yb, yd, None))[7:].tolist() == pytest.approx(
        oracle.em_ratio(b64[0], b64[1])[7:].tolist(), rel=1e-6)


def test_autograd_em_update_equals_fused_step():
    """The differentiable EM update (A, the ratio kernel, A', the update kernel)
    computes, step for step, the arithmetic of the fused regularised EM step:
    bitwise the same image."""
    from paper_2301_09710_gb300.autograd import em_update
    prob, ang = _small()
    plan = make_plan(prob, ang, "fused")
    psf = oracle_psf(prob, "fused")
    y = synthetic.poisson_counts(oracle.forward(prob.x, prob.mu, psf, prob.dy, ang) * 50, 2)
    rbar = np.full_like(y, 0.1 * y.mean())
    x0 = np.where(prob.body, 1.0, 0.0).astype(np.float32) + 0.1
    u = np.random.default_rng(4).uniform(0.2, 3.0, x0.shape).astype(np.float32)
    s = plan.sensitivity()
    for beta in (0.0, 0.05, 5.0):
        xg = dev(x0)
        plan.em_step_reg(xg, dev(y), dev(u), beta, rbar=dev(rbar), niter=1)
        with torch.no_grad():
            xa = em_update(dev(x0), dev(y), dev(rbar), plan, s, dev(u), beta)
        assert np.array_equal(host(xa), host(xg)), f"beta={beta}"
    plan.check()
